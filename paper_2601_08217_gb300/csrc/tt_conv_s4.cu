// Samples-per-thread = 4 variants of the tiled FP32 channel kernel, 128 threads per CTA (one TU per S).
#include "tt_conv_kernel.cuh"

cudaError_t tt_launch_conv_s4(const TTLaunch &L, cudaStream_t st) { return tt::tt_launch_spt<4, false, TT_TPB>(L, st); }
