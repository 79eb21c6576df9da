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

cudaError_t build_pass3_ids(pcx_ctx* c) {
  if (!c->dev.mid || c->dev.mid3) return cudaSuccess;
  const int n = c->n;
  if (n != 32 && n != 64 && n != 128) return cudaSuccess;
  cudaError_t e = cudaMalloc(&c->dev.mid3, (size_t)n * n * n * 4);
  if (e != cudaSuccess) return e;
  e = n == 32 ? fftk::build_pass3_ids_n<32>(c->dev.mid, c->dev.mid3, nullptr)
              : (n == 64 ? fftk::build_pass3_ids_n<64>(c->dev.mid, c->dev.mid3, nullptr)
                         : fftk::build_pass3_ids_n<128>(c->dev.mid, c->dev.mid3, nullptr));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e;
}
}  // namespace pcx
