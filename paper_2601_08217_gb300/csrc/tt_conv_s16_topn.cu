// Samples-per-thread = 16 variants of the tiled FP32 channel kernel with sparse convolution
// (top-n taps per symbol and link, Sec. III-C), 128 threads per CTA; one TU per S.
#include "tt_conv_kernel.cuh"

cudaError_t tt_launch_conv_s16_topn(const TTLaunch &L, cudaStream_t st) { return tt::tt_launch_spt<16, true, TT_TPB>(L, st); }
