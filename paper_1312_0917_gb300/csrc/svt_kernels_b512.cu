// svt_kernels_b512.cu -- the persistent kernel built at 512 threads per CTA
// (namespace svt::b512), one of the block sizes svt_autotune chooses from.
#define SVT_BLOCK 512
#include "svt_kernels.cu"
