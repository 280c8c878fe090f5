// The record pass of the forward preprocess (the second of its two kernels; see
// preprocess_fwd.cuh), one instantiation per storage type pair, with and without the appearance
// transform. A translation unit of its own so that it compiles in parallel with preprocess.cu.
#include "preprocess_fwd.cuh"

namespace gsr {
namespace {

template <typename AT, typename ST>
void launch_rec_t(const GaussArgs& g, const CamBatch& cams, float eps, int aa, const PreOut& out, int blocks,
                  cudaStream_t s) {
  if (g.mlp || g.mlp_cached)
    preprocess_rec_kernel<AT, ST, true><<<blocks, kPreThreads, 0, s>>>(g, cams, eps, aa, out);
  else
    preprocess_rec_kernel<AT, ST, false><<<blocks, kPreThreads, 0, s>>>(g, cams, eps, aa, out);
}

}  // namespace

void launch_preprocess_rec(const GaussArgs& g, const CamBatch& cams, float eps2d, int antialiased,
                           const PreOut& out, int rec_blocks, cudaStream_t s) {
  if (rec_blocks <= 0) return;
#define GSR_PRE(AT, ST) launch_rec_t<AT, ST>(g, cams, eps2d, antialiased, out, rec_blocks, s)
  if (g.attr_dtype == 0 && g.sh_dtype == 0) GSR_PRE(float, float);
  else if (g.attr_dtype == 0 && g.sh_dtype == 1) GSR_PRE(float, __half);
  else if (g.attr_dtype == 0 && g.sh_dtype == 2) GSR_PRE(float, __nv_bfloat16);
  else if (g.attr_dtype == 1 && g.sh_dtype == 1) GSR_PRE(__half, __half);
  else if (g.attr_dtype == 2 && g.sh_dtype == 2) GSR_PRE(__nv_bfloat16, __nv_bfloat16);
  else if (g.attr_dtype == 1 && g.sh_dtype == 0) GSR_PRE(__half, float);
  else if (g.attr_dtype == 2 && g.sh_dtype == 0) GSR_PRE(__nv_bfloat16, float);
  else if (g.attr_dtype == 1 && g.sh_dtype == 2) GSR_PRE(__half, __nv_bfloat16);
  else GSR_PRE(__nv_bfloat16, __half);
#undef GSR_PRE
}

}  // namespace gsr
