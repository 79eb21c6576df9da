// complex64 instantiation of the apply and preconditioner kernels.
#include "fft3_kernels.cuh"

namespace pcx {
template cudaError_t run_apply_t<float>(const pcx_ctx*, const KParams&, const void*, void*, int, int, void*,
                                        const KParams*, int, cudaStream_t, bool);
template cudaError_t run_precond_t<float>(const pcx_ctx*, const KParams&, const void*, void*, int, cudaStream_t);
template cudaError_t run_div_norms_t<float>(const pcx_ctx*, const KParams&, const void*, int, double*,
                                            cudaStream_t);
template cudaError_t run_fft_t<float>(const pcx_ctx*, const void*, void*, int, int, cudaStream_t);
template cudaError_t run_curl_h_t<float>(const pcx_ctx*, const KParams&, const void*, void*, int, int, cudaStream_t);
template cudaError_t run_curl_add_t<float>(const pcx_ctx*, const KParams&, const void*, const void*, void*, int, double, int,
                                        cudaStream_t);
template cudaError_t run_eps_cells_t<float>(const pcx_ctx*, const void*, const void*, void*, int, double, cudaStream_t);
}  // namespace pcx
