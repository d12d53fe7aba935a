"""FP64 CPU oracle for the McKernel / Fastfood feature map (arXiv 1702.08159).

This package is TEST INFRASTRUCTURE. Only the test suite, the package smoke
check (``__graft_entry__.smoke``) and the CPU-baseline leg of ``bench.py`` may
import it. The product path (the CUDA library and its Python binding) never
imports, links or executes anything here, and nothing here imports the product
path: the two share no code. The only module both sides use is the seeded
input generator (``workloads.py`` at the repository root), which holds none of
the method's arithmetic.

Everything is written from the paper's definitions in plain numpy, float64,
with no blocking, fusion or reordering beyond what the definitions state:

* ``philox``   -- Philox4x32-10 counter-based generator (Salmon et al., SC'11),
                  the hash that replaces Murmurhash in Sec. "McKernel" (B, Pi, G).
* ``fastfood`` -- the Hadamard recursion (Sec. "Fast Walsh Hadamard"), the
                  random diagonal/permutation tables (Sec. "McKernel": B, H, Pi,
                  G, C; Sec. "Customizing McKernel" for the Matern C), the map
                  Z = (1/(sigma sqrt n)) C H G Pi H B (Eq. etn:mckernel) and the
                  feature map [cos(Zx), sin(Zx)] (Eq. etn:mcfeatures).
* ``training`` -- softmax(W phi + b) (Sec. "Empirical Analysis"), the
                  cross-entropy loss (the multi-class form of Eq. etn:loss) and
                  its gradients by the chain rule, plus central finite
                  differences.

Parity status of each function is stated in its module header.
"""
