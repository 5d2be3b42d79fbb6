// svt_kernels_b128.cu -- the persistent kernel built at 128 threads per CTA
// (namespace svt::b128), one of the block sizes svt_autotune chooses from.
#define SVT_BLOCK 128
#include "svt_kernels.cu"
