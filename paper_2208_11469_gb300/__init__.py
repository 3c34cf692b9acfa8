"""GB300-native ProbGraph hot path: sketch construction and sketched
|N(u) ∩ N(v)| estimation over int32 CSR graphs, as CUDA kernels behind a
C ABI (include/pg.h). The compiled library is loaded on first use by
`paper_2208_11469_gb300.pg`; importing this package loads nothing."""
