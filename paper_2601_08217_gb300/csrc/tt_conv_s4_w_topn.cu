// Samples-per-thread = 4 variants of the tiled FP32 channel kernel with sparse convolution
// (top-n taps per symbol and link, Sec. III-C), 256 threads per CTA; one TU per S.
#include "tt_conv_kernel.cuh"

cudaError_t tt_launch_conv_s4_w_topn(const TTLaunch &L, cudaStream_t st) { return tt::tt_launch_spt<4, true, TT_TPB_WIDE>(L, st); }
