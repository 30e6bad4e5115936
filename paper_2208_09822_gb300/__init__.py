"""GB300 small-GEMM library after IAAT (arXiv 2208.09822).

C = alpha*op(A)*op(B) + beta*C for batches of small FP32/FP64 instances,
computed by CUDA kernels for sm_103a behind a C ABI (include/iaat.h).  The
Python layer (``iaat``) only marshals arguments into that ABI.
"""
