"""GB300-native subspace multicoil NUFFT operator of StoDIP (arXiv 2408.02367).

A_c(x)[j] = NUFFT_{omega_j}(S_c * sum_k V[t_j, k] x_k) and its adjoint, computed by
hand-written sm_103a CUDA kernels behind a C ABI (include/stodip_op.h).  The
binding (`paper_2408_02367_gb300.op`) loads the library lazily so that the input
generators in `synth` import without a GPU.
"""
__all__ = ["synth"]
