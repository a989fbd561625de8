// Forward apply kernels instantiated for interpolation orders Ps = 3, Pang = 5.
#include "fwd_kernels.cuh"

namespace ifgf {
template ifgf_status prepare_t<3, 5>(Plan &, cudaStream_t);
template ifgf_status run_apply_t<3, 5>(Plan &, const void *, void *, int, int, cudaStream_t);
template ifgf_status run_adjoint_t<3, 5>(Plan &, const void *, void *, int, int, cudaStream_t, void *, void *,
                                              void **, void *const *, double *);
template ifgf_status run_dk_t<3, 5>(Plan &, int, int, cudaStream_t, const void *, void **, double *,
                                         long long *);
template ifgf_status run_far_t<3, 5>(Plan &, const double *, long long, void *, int, int, cudaStream_t);
}  // namespace ifgf
