// Internal declarations of the pcx library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pcx.h"

namespace pcx {

using cd = std::complex<double>;

// Per-k scalars every Fourier-space kernel needs.  The mode symbol is
//   kappa_i(p) = sum_j b[j][i] * (L1[p_j] + i kt[j] L0[p_j]) + i kq[i] L0[p_i]
// (kq = 0 for the summed reading, kt = 0 and kq = k for the literal reading,
// where the S_j table keeps only L1).  See pcx_symbols in pcx.h.
struct KParams {
  double b[9];      // b = A^{-1}, row-major: b[3*j + i] = b_ji
  double kt[3];     // coefficient of i Lambda_0 inside S_j
  double kq[3];     // coefficient of i Lambda_0(p_i) added to kappa_i
  double gamma;     // penalty coefficient (per-mode form: its scale, see per_mode)
  int diag_b;       // 1 when b is diagonal (simple cubic fast path)
  int per_mode;     // penalty form: 0 scalar; 1 gamma_p = gamma max(1, 1/|kappa_p|^2);
                    // 2 gamma_p = gamma / |kappa_p|^2 (gamma times the longitudinal projector)
};

// Kernel variants of the three-pass chain (fft3_kernels.cuh): x passes
// 0..X3_VARIANTS-1, z pass 0..Z3_VARIANTS-1, and the build-time defaults
// used when neither the caller nor the autotuner chose.
constexpr int X3_VARIANTS = 4, Z3_VARIANTS = 2;
#ifndef PCX_X3_VARIANT
#define PCX_X3_VARIANT 3
#endif
#ifndef PCX_Z3_VARIANT
#define PCX_Z3_VARIANT 0
#endif

// Device-resident, k-independent tables of one context.
struct DeviceTables {
  void* lam64 = nullptr;   // [2][N] double2: Lambda_1, Lambda_0
  void* lam32 = nullptr;   // [2][N] float2
  void* tw64 = nullptr;    // [N] double2: exp(-2 pi i m / N)
  void* tw32 = nullptr;    // [N] float2
  // M as material ids: one uchar4 per cell (materials at E1, E2, E3 and the
  // volume centre) plus a per-material table of the nine block entries.
  void* mid = nullptr;     // [N^3] uchar4
  void* mtab64 = nullptr;  // [n_mat][9] double: e11 e22 e33 re12 im12 re13 im13 re23 im23
  void* mtab32 = nullptr;  // [n_mat][9] float
  void* mtab12 = nullptr;  // [n_mat][12] float: e11 e22 e33 0 re12 im12 re13 im13 re23 im23 0 0 (16-byte records)
  int n_mat = 0;
  void* mid3 = nullptr;    // [N^3] uchar4: mid in the order of the three-pass z tiles (N = 32, 64, 128)
  // M as dense blocks (caller-supplied cell blocks, or more than 255 materials)
  void* m64 = nullptr;     // [9][N^3] double: d1 d2 d3 re12 im12 re13 im13 re23 im23
  void* m32 = nullptr;     // [9][N^3] float
};

}  // namespace pcx

struct pcx_ctx {
  int n = 0;
  int m = 1;
  int reading = PCX_CT_SUMMED;
  int m_kind = PCX_M_TRIVIAL;   // discrete inverse permittivity of the apply
  int device = 0;
  double A[9] = {0};
  double b[9] = {0};
  std::vector<pcx::cd> lam1, lam0;       // host copies of the symbol tables
  std::vector<double> blocks;            // host N^3 x 9 packed cell blocks
  double lambda_min = 0.0;
  pcx::DeviceTables dev;
  // apply tuning and scratch: vectors per L2-resident chunk (0 = from L2 size)
  int apply_chunk = 0;
  // apply pass structure: PCX_APPLY_AUTO, PCX_APPLY_FIVE_PASS or PCX_APPLY_THREE_PASS
  int apply_path = 0;
  // kernel variants of the three-pass chain's x and z passes (-1: build default)
  int x3_variant = -1, z3_variant = -1;
  void* scratch = nullptr;     // gamma kappa.x carried from pass 1 to pass 5
  size_t scratch_bytes = 0;
  size_t l2_bytes = 0;
  // k table of the k-batched apply (device, grown on demand)
  void* ktab = nullptr;
  size_t ktab_bytes = 0;
  // CUDA graphs of the apply launch chain (fft_apply.cu), when enabled
  int use_graphs = 0;
  void* graphs = nullptr;
  int cnn_form = 0;   // PCX_CNN_HERMITIAN | PCX_CNN_BF16 flags
  int penalty_form = 0;   // PCX_PENALTY_SCALAR, PCX_PENALTY_PER_MODE or PCX_PENALTY_PROJECTOR
  // staging for pcx_apply_host: two slots of X and Y chunks, copy streams
  // and slot events (created on first use)
  void* stage_x = nullptr;
  void* stage_y = nullptr;
  size_t stage_bytes = 0;       // bytes of the two slots together, per buffer
  cudaStream_t copy_stream[2] = {nullptr, nullptr};   // host->device, device->host
  // streams of the k-points that pcx_solve runs at the same time (created on first use)
  std::vector<cudaStream_t> solve_streams;
  cudaEvent_t slot_event[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
  std::string err;
};

namespace pcx {

// setup.cpp
pcx_status validate_desc(const pcx_setup_desc* d, std::string& err);
pcx_status sample_blocks(const pcx_setup_desc* d, const double* A, std::vector<double>& blocks,
                         std::vector<int32_t>* ids, std::string& err);
long long first_non_hpd(const std::vector<double>& blocks);
long long crossdof_unproven(int n, int n_mat, const double* eps, const std::vector<int32_t>& ids, std::string* why);
pcx_status setup_context(const pcx_setup_desc* d, pcx_ctx* c);
KParams make_kparams(const pcx_ctx* c, const double k[3], double gamma);
double gamma_rule(const double k[3]);

// kernels (fft_apply.cu, blas.cu)
// curl-sandwich approximate inverse T0 (W may be R) on the five-pass chain of
// the apply, with the context-owned scratch
cudaError_t launch_t0(pcx_ctx* c, const KParams& kp, const void* R, void* W, int nvec, int precision, cudaStream_t s);
// apply with the context-owned scratch (allocated on first use / growth)
cudaError_t launch_apply(pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec, int precision,
                         cudaStream_t s);
// T0 with caller-provided scratch of apply_scratch_bytes(c, precision, nvec) bytes
cudaError_t launch_t0_scratch(const pcx_ctx* c, const KParams& kp, const void* R, void* W, int nvec, int precision,
                              void* scratch, cudaStream_t s);
// apply with caller-provided scratch of apply_scratch_bytes(c, precision, nvec) bytes
cudaError_t launch_apply_scratch(const pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec,
                                 int precision, void* scratch, cudaStream_t s);
// apply with the file-scope device scratch (pcx_apply_noalloc); returns
// cudaErrorInvalidValue if one vector's scratch exceeds PCX_NOALLOC_SCRATCH_BYTES
cudaError_t launch_apply_noalloc(const pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec,
                                 int precision, cudaStream_t s);
int apply_chunk(const pcx_ctx* c, int precision);
// pass structure the apply runs: PCX_APPLY_FIVE_PASS, PCX_APPLY_THREE_PASS, or 7 (M_CrossDoF)
int effective_apply_path(const pcx_ctx* c, int precision);
// dev.mid3 from dev.mid (allocates; a no-op where the three-pass form does not exist)
cudaError_t build_pass3_ids(pcx_ctx* c);
// k-batched apply: nk groups of vec_per_k vectors, group i at kps_host[i]
cudaError_t launch_apply_kbatch(pcx_ctx* c, const KParams* kps_host, int nk, int vec_per_k, const void* X, void* Y,
                                int precision, cudaStream_t s);
// release the graph cache of a context
void free_apply_graphs(pcx_ctx* c);
// tune.cpp
cudaError_t autotune_apply(pcx_ctx* c, int precision, int nvec, cudaStream_t s, pcx_tune_result* out);
size_t apply_scratch_bytes(const pcx_ctx* c, int precision, int nvec);
cudaError_t launch_precond(const pcx_ctx* c, const KParams& kp, const void* R, void* W, int nvec,
                           int precision, cudaStream_t s);
// learned correction of K_P^{-1} (learned.cpp; parameters: cnn::NPARAMS floats)
cudaError_t cnn_gates(pcx_ctx* c, const float* params, float* gates, cudaStream_t s);
cudaError_t cnn_forward(pcx_ctx* c, const float* params, const float* gates, const void* U, void* Y, int nvec,
                        cudaStream_t s);
cudaError_t cnn_grad(pcx_ctx* c, const float* params, const void* U, const void* T, const double* wv_host, int nvec,
                     float* grad, int accumulate, double* loss_host, cudaStream_t s);
cudaError_t cnn_precond(pcx_ctx* c, const KParams& kp, const float* params, const float* gates, const void* R, void* W,
                        int nvec, cudaStream_t s);
cudaError_t cnn_pairs(pcx_ctx* c, const KParams& kp, const void* R, const void* E, void* U, void* T, double* enorm2_host,
                      int nvec, cudaStream_t s);
cudaError_t cg_solve(pcx_ctx* c, const KParams& kp, const void* R, void* E, int nvec, double tol, int maxit,
                     int* iters, double* relres, cudaStream_t s);
// pieces of the curl-sandwich approximate inverse (fft_kernels.cuh):
// U = K_A^H X / |k|^(2 pow);  Y (+)= s K_A Wm / |k|^2 [+ conj(kappa)(kappa.R)/(gamma |k|^4)];
// Mo = s (M^{-1} E + Add) per cell (real space)
cudaError_t launch_curl_h(const pcx_ctx* c, const KParams& kp, const void* X, void* U, int nvec, int pow, int precision,
                          cudaStream_t s);
cudaError_t launch_curl_add(const pcx_ctx* c, const KParams& kp, const void* Wm, const void* R, void* Y, int nvec,
                            double scale, int accumulate, int precision, cudaStream_t s);
cudaError_t launch_eps_cells(const pcx_ctx* c, const void* E, const void* Add, void* Mo, int nvec, double scale,
                             int precision, cudaStream_t s);
// T0 R (learned.cpp), workspace from the context
cudaError_t sandwich_precond(pcx_ctx* c, const KParams& kp, const void* R, void* W, int nvec, int precision,
                             cudaStream_t s);
// unnormalised 3D DFT of every component, dir > 0: N^{3/2} F3_3, dir < 0: N^{3/2} F3_3^H (Y may be X)
cudaError_t launch_fft(const pcx_ctx* c, const void* X, void* Y, int nvec, int dir, int precision, cudaStream_t s);
// out[v] = x_v^H K_B x_v, out[nvec + v] = ||x_v||^2 (device doubles, zeroed here)
cudaError_t launch_div_norms(const pcx_ctx* c, const KParams& kp, const void* X, int nvec, int precision, double* out,
                             cudaStream_t s);
// Gram G = A^H B.  complex128: double-float sums (gram_x.cu).  complex64:
// the FP32-pipe kernel of gram_cc.cu or the tensor-core kernel of gram_tc.cu
// as set_gram_path chooses (0: by shape, 1: tensor cores, 2: FP32 pipes),
// the generic CUDA-core kernel of blas.cu where neither applies
cudaError_t launch_gram(const void* A, int na, const void* B, int nb, size_t L, int precision,
                        double* G, cudaStream_t s);
cudaError_t launch_gram_cuda_cores(const void* A, int na, const void* B, int nb, size_t L, int precision,
                                   double* G, cudaStream_t s);
bool gram_tc_supported(int na, int nb, size_t L);
bool gram_cc_supported(const void* A, const void* B, int na, int nb, size_t L);
cudaError_t launch_gram_cc(const void* A, int na, const void* B, int nb, size_t L, double* G, cudaStream_t s);
void set_gram_path(int path);
// free the per-stream partial-sum buffers of the Gram kernels for stream s
void gram_cc_release_stream(cudaStream_t s);
void gram_tc_release_stream(cudaStream_t s);
void gram_x_release_stream(cudaStream_t s);
void cnn_release_stream(cudaStream_t s);
int get_gram_path();
// G = [A1 | A2]^H B: A1 (na1 columns) and A2 (na2 columns) complex128, B
// complex64; double-float accumulation on the FP32 pipes.
cudaError_t launch_gram_x(const void* A1, int na1, const void* A2, int na2, const void* B, int nb, size_t L,
                          double* G, cudaStream_t s);
// G = A^H B with A, B complex128, double-float sums on the FP32 pipes
cudaError_t launch_gram_dd(const void* A, int na, const void* B, int nb, size_t L, double* G, cudaStream_t s);
cudaError_t launch_gram_tc(const void* A, int na, const void* B, int nb, size_t L, double* G, cudaStream_t s);
cudaError_t launch_combine(const void* S, int ns, const double* C, int ny, double beta, void* Y,
                           size_t L, int precision, cudaStream_t s);
// Y64 += S32 C (complex64 combination evaluated in FP32, added into complex128)
cudaError_t launch_combine_add32(const void* S32, int ns, const double* C, int ny, void* Y64, size_t L,
                                cudaStream_t s);
cudaError_t launch_residual(const void* X, const void* AX, const double* theta, void* R,
                            double* norms, int nvec, size_t L, int precision, cudaStream_t s);
// complex128 X, AX -> complex64 R = AX - X theta and X, FP64 norms (the
// mixed-precision refinement's residual)
cudaError_t launch_residual_mixed(const void* X, const void* AX, const double* theta, void* R32, void* X32,
                                  double* norms, int nvec, size_t L, cudaStream_t s);
cudaError_t launch_fill_random(void* X, int nvec, size_t L, uint64_t seed, int precision,
                               cudaStream_t s);
cudaError_t launch_deflate_p0(void* X, int nvec, int n, int precision, cudaStream_t s);
cudaError_t launch_convert(const void* src, int src_prec, void* dst, int dst_prec, size_t count,
                           cudaStream_t s);

// solver.cpp
pcx_status solve(pcx_ctx* c, const double* kpts, int nk, int nev, double tol,
                 const pcx_solve_opts* opts, double* eig_out, double* res_out, int* iters_out,
                 void* vec_out, cudaStream_t s);

inline bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Raise the dynamic shared-memory limit of a kernel (on the current device)
// to at least `bytes`.  The limit is a property of the kernel, shared by
// every thread that launches it, so it only ever grows: a launch sized
// under the limit stays valid when another thread raises it (several
// k-points of pcx_solve in flight launch the same kernels with different
// sizes).
cudaError_t raise_dyn_smem(const void* func, size_t bytes);

}  // namespace pcx
