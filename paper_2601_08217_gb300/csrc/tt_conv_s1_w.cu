// Samples-per-thread = 1 variants of the tiled FP32 channel kernel, 256 threads per CTA (one TU per S).
#include "tt_conv_kernel.cuh"

cudaError_t tt_launch_conv_s1_w(const TTLaunch &L, cudaStream_t st) { return tt::tt_launch_spt<1, false, TT_TPB_WIDE>(L, st); }
