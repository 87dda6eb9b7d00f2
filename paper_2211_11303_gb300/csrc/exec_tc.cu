// The FP32 task executor with TF32 tensor-core tile products (HLU_TF32
// factorisations), built from exec.cu in namespace hlu::tcx.  Its kernel
// allocates tensor memory, which holds it to one CTA per SM; the plain FP32
// and FP64 executors (exec.cu) keep two.
#define HLU_EXEC_TC 1
#include "exec.cu"
