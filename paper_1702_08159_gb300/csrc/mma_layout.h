// Element orders of the tensor-core feature kernel at d = 1024 (host and
// device). A warp holds a vector as chunk registers j = 0..31 of 32 lanes, in
// the fragment order of mma_h16.cuh: register j = (tile, r, h) with
// tile = j / 8, r = (j / 2) % 4, h = j % 2, lane = 4 g + t; the fragment
// (row, col) = (g + 8 (r & 1), 2 t + 8 (r >> 1) + h) of tile `tile`.
// Input order (the A operand of the first product): element
// tile * 256 + 16 row + col. Output order (after the two digits): element
// tile * 256 + 16 col + row.
#pragma once

namespace mck {

__host__ __device__ constexpr int mma_row(int lane, int j) { return (lane >> 2) + 8 * ((j >> 1) & 1); }
__host__ __device__ constexpr int mma_col(int lane, int j) {
  return 2 * (lane & 3) + 8 * ((j >> 2) & 1) + (j & 1);
}
__host__ __device__ constexpr int mma_in(int lane, int j) {
  return (j >> 3) * 256 + 16 * mma_row(lane, j) + mma_col(lane, j);
}
__host__ __device__ constexpr int mma_out(int lane, int j) {
  return (j >> 3) * 256 + 16 * mma_col(lane, j) + mma_row(lane, j);
}
// Lane and register holding element s in the output order.
__host__ __device__ constexpr int mma_out_lane(int s) {
  return 4 * ((s & 15) & 7) + ((((s >> 4) & 15) >> 1) & 3);
}
__host__ __device__ constexpr int mma_out_reg(int s) {
  return (s >> 8) * 8 + 2 * (2 * (((s >> 4) & 15) >> 3) + ((s & 15) >> 3)) + (((s >> 4) & 15) & 1);
}

}  // namespace mck
