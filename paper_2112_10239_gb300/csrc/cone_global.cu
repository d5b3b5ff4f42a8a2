// The global-memory tier of the cone kernel (cone_kernel<real, GRAD, true>: windows whose
// psi and lambda do not fit in shared memory) in a translation unit of its own, so that it
// keeps the default ptxas optimisation level while cone.cu's shared-memory tier takes -O1.
// Emits launch_cone_global and launch_batch_global, which cone.cu's launchers call.
#define TLQ_CONE_GLOBAL_TU
#include "cone.cu"
