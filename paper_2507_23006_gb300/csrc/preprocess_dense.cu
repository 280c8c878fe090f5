// The forward preprocess for launches where many Gaussians survive the culls (a street-level
// view, a dense scene): three resident blocks per SM, leaving the per-record work its registers.
// A translation unit of its own so that the two sets of instantiations compile in parallel.
#include "preprocess_fwd.cuh"

namespace gsr {
namespace {

template <typename AT, typename ST>
void launch_dense_t(const GaussArgs& g, const CamBatch& cams, float eps, int aa, const PreOut& out, int blocks,
                    cudaStream_t s) {
  if (g.mlp || g.mlp_cached)
    preprocess_fwd_kernel<AT, ST, true, 3><<<blocks, kPreThreads, 0, s>>>(g, cams, eps, aa, out);
  else
    preprocess_fwd_kernel<AT, ST, false, 3><<<blocks, kPreThreads, 0, s>>>(g, cams, eps, aa, out);
}

}  // namespace

void launch_preprocess_fwd_dense(const GaussArgs& g, const CamBatch& cams, float eps2d, int antialiased,
                                 const PreOut& out, int blocks, cudaStream_t s) {
#define GSR_PRE(AT, ST) launch_dense_t<AT, ST>(g, cams, eps2d, antialiased, out, blocks, s)
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
