// extern "C" entry points of libpcx (declared in include/pcx.h): argument
// validation, error strings and dispatch to the setup code, the kernels and
// the solver.  Invalid arguments are rejected here, before any launch.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "cnn.h"
#include "linalg.h"
#include "pcx_internal.h"

namespace {

thread_local std::string g_err;   // errors raised without a context

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

pcx_status cuda_fail(pcx_ctx* c, const char* where, cudaError_t e) {
  std::string msg = std::string(where) + ": CUDA error " + cudaGetErrorString(e);
  if (c) c->err = msg;
  else g_err = msg;
  return e == cudaErrorMemoryAllocation ? PCX_ENOMEM : PCX_ECUDA;
}

pcx_status inval(pcx_ctx* c, const std::string& msg) {
  if (c) c->err = msg;
  else g_err = msg;
  return PCX_EINVAL;
}

bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + nb && y < x + na;
}

}  // namespace

extern "C" {

pcx_status pcx_setup(const pcx_setup_desc* desc, pcx_ctx** out) {
  if (!desc || !out) return inval(nullptr, "pcx_setup: NULL argument");
  *out = nullptr;
  pcx_ctx* c = new (std::nothrow) pcx_ctx();
  if (!c) {
    g_err = "pcx_setup: out of host memory";
    return PCX_ENOMEM;
  }
  pcx_status st;
  try {
    st = pcx::setup_context(desc, c);
  } catch (const std::bad_alloc&) {
    c->err = "pcx_setup: out of host memory";
    st = PCX_ENOMEM;
  }
  if (st == PCX_OK || st == PCX_ENOTHPD) {
    *out = c;
    return st;
  }
  g_err = c->err;
  pcx_destroy(c);
  return st;
}

pcx_status pcx_sample_host(const pcx_setup_desc* desc, double* blocks_out, int32_t* ids_out, long long* first_bad) {
  if (!desc || !blocks_out) return inval(nullptr, "pcx_sample_host: NULL argument");
  std::string err;
  pcx_status st = pcx::validate_desc(desc, err);
  if (st != PCX_OK) return inval(nullptr, err);
  std::vector<double> blocks;
  std::vector<int32_t> ids;
  try {
    st = pcx::sample_blocks(desc, desc->lattice, blocks, (ids_out || desc->m_kind == PCX_M_CROSSDOF) ? &ids : nullptr,
                            err);
  } catch (const std::bad_alloc&) {
    g_err = "pcx_sample_host: out of host memory";
    return PCX_ENOMEM;
  }
  if (st != PCX_OK) {
    g_err = err;
    return st;
  }
  std::memcpy(blocks_out, blocks.data(), blocks.size() * sizeof(double));
  if (ids_out) std::memcpy(ids_out, ids.data(), ids.size() * sizeof(int32_t));
  if (first_bad)
    *first_bad = desc->m_kind == PCX_M_CROSSDOF ? pcx::crossdof_unproven(desc->n, desc->n_mat, desc->eps, ids, nullptr)
                                                : pcx::first_non_hpd(blocks);
  return PCX_OK;
}

void pcx_destroy(pcx_ctx* c) {
  if (!c) return;
  pcx::free_apply_graphs(c);
  for (auto& st : c->copy_stream)
    if (st) cudaStreamDestroy(st);
  for (cudaStream_t st : c->solve_streams) {
    pcx::gram_cc_release_stream(st);
    pcx::gram_tc_release_stream(st);
    pcx::gram_x_release_stream(st);
    pcx::cnn_release_stream(st);
    cudaStreamDestroy(st);
  }
  for (auto& row : c->slot_event)
    for (auto& ev : row)
      if (ev) cudaEventDestroy(ev);
  void* ptrs[] = {c->dev.lam64, c->dev.lam32, c->dev.tw64,  c->dev.tw32, c->dev.m64,  c->dev.m32,
                  c->dev.mid,   c->dev.mtab64, c->dev.mtab32, c->scratch, c->stage_x, c->stage_y, c->ktab,
                  c->dev.mid3, c->dev.mtab12};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete c;
}

const char* pcx_last_error(const pcx_ctx* c) { return c ? c->err.c_str() : g_err.c_str(); }

int pcx_grid_n(const pcx_ctx* c) { return c ? c->n : 0; }

size_t pcx_vector_length(const pcx_ctx* c) { return c ? (size_t)3 * c->n * c->n * c->n : 0; }

pcx_status pcx_cell_blocks(const pcx_ctx* c, double* host_out, double* lambda_min) {
  if (!c || c->blocks.empty()) return inval(const_cast<pcx_ctx*>(c), "pcx_cell_blocks: no context");
  if (host_out) std::memcpy(host_out, c->blocks.data(), c->blocks.size() * sizeof(double));
  if (lambda_min) {
    // smallest eigenvalue of every Hermitian cell block (Jacobi on 3x3)
    double lo = INFINITY;
    const size_t n3 = c->blocks.size() / 9;
    for (size_t i = 0; i < n3; ++i) {
      const double* b = &c->blocks[9 * i];
      std::vector<pcx::cd> a = {b[0], {b[3], b[4]}, {b[5], b[6]}, {b[3], -b[4]}, b[1], {b[7], b[8]},
                                {b[5], -b[6]}, {b[7], -b[8]}, b[2]};
      std::vector<double> w;
      std::vector<pcx::cd> v;
      pcx::herm_eig(3, a, w, v);
      lo = std::min(lo, w[0]);
    }
    *lambda_min = lo;
  }
  return PCX_OK;
}

pcx_status pcx_symbols(const pcx_ctx* c, const double k[3], double gamma, double* s_tab, double* q_tab, double* b,
                       double* gamma_out) {
  if (!c || !k) return inval(const_cast<pcx_ctx*>(c), "pcx_symbols: NULL argument");
  pcx::KParams kp = pcx::make_kparams(c, k, gamma);
  const int n = c->n;
  for (int j = 0; j < 3; ++j)
    for (int p = 0; p < n; ++p) {
      const pcx::cd l1 = c->lam1[p], l0 = c->lam0[p];
      const pcx::cd s = l1 + pcx::cd(0, kp.kt[j]) * l0;
      const pcx::cd q = pcx::cd(0, kp.kq[j]) * l0;
      if (s_tab) {
        s_tab[2 * (j * n + p)] = s.real();
        s_tab[2 * (j * n + p) + 1] = s.imag();
      }
      if (q_tab) {
        q_tab[2 * (j * n + p)] = q.real();
        q_tab[2 * (j * n + p) + 1] = q.imag();
      }
    }
  if (b) std::memcpy(b, c->b, 9 * sizeof(double));
  if (gamma_out) *gamma_out = kp.gamma;
  return PCX_OK;
}

static pcx_status check_block(pcx_ctx* c, const char* who, const void* X, const void* Y, int nvec, int precision) {
  if (!c) return inval(nullptr, std::string(who) + ": NULL context");
  if (precision != PCX_FP64 && precision != PCX_FP32) return inval(c, std::string(who) + ": bad precision");
  if (nvec < 0) return inval(c, std::string(who) + ": nvec < 0");
  if (nvec == 0) return PCX_OK;
  if (!X || !Y) return inval(c, std::string(who) + ": NULL buffer");
  if (!aligned16(X) || !aligned16(Y)) return inval(c, std::string(who) + ": buffers must be 16-byte aligned");
  return PCX_OK;
}

pcx_status pcx_set_apply_chunk(pcx_ctx* c, int chunk) {
  if (!c) return inval(nullptr, "pcx_set_apply_chunk: NULL context");
  c->apply_chunk = chunk > 0 ? chunk : 0;
  return PCX_OK;
}

int pcx_get_apply_chunk(const pcx_ctx* c, int precision) { return c ? pcx::apply_chunk(c, precision) : 0; }

pcx_status pcx_apply(pcx_ctx* c, const double k[3], double gamma, const void* X, void* Y, int nvec, int precision,
                     void* stream) {
  pcx_status st = check_block(c, "pcx_apply", X, Y, nvec, precision);
  if (st != PCX_OK || nvec == 0) return st;
  if (!k) return inval(c, "pcx_apply: NULL k");
  const size_t bytes = pcx_vector_length(c) * nvec * (precision == PCX_FP64 ? 16 : 8);
  if (ranges_overlap(X, bytes, Y, bytes)) return inval(c, "pcx_apply: X and Y overlap");
  pcx::KParams kp = pcx::make_kparams(c, k, gamma);
  cudaError_t e = pcx::launch_apply(c, kp, X, Y, nvec, precision, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_apply", e);
}

pcx_status pcx_apply_noalloc(pcx_ctx* c, const double k[3], double gamma, const void* X, void* Y, int nvec,
                             int precision, void* stream) {
  pcx_status st = check_block(c, "pcx_apply_noalloc", X, Y, nvec, precision);
  if (st != PCX_OK || nvec == 0) return st;
  if (!k) return inval(c, "pcx_apply_noalloc: NULL k");
  // one vector's scratch: N^3 entries of gamma kappa.x, and for M_CrossDoF
  // the real-space field of its stencil pass (3 N^3 more)
  const bool crossdof = c->m_kind == PCX_M_CROSSDOF;
  const size_t per_vec = (size_t)c->n * c->n * c->n * (precision == PCX_FP64 ? 16 : 8) * (crossdof ? 4 : 1);
  if (per_vec > (size_t)PCX_NOALLOC_SCRATCH_BYTES)
    return inval(c, std::string("pcx_apply_noalloc: the scratch of one vector (") + std::to_string(per_vec) +
                        (crossdof ? " bytes: 4 N^3 entries for M_CrossDoF" : " bytes: N^3 entries") +
                        ") exceeds the 32 MiB static scratch; use pcx_apply");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device)
    return inval(c, "pcx_apply_noalloc: the context's device " + std::to_string(c->device) +
                        " is not the current device " + std::to_string(dev));
  const size_t bytes = pcx_vector_length(c) * nvec * (precision == PCX_FP64 ? 16 : 8);
  if (ranges_overlap(X, bytes, Y, bytes)) return inval(c, "pcx_apply_noalloc: X and Y overlap");
  pcx::KParams kp = pcx::make_kparams(c, k, gamma);
  cudaError_t e = pcx::launch_apply_noalloc(c, kp, X, Y, nvec, precision, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_apply_noalloc", e);
}

// The host-buffer pipeline of pcx_apply_host and pcx_apply_kbatch_host:
// nk groups of vpk vectors, group g applied with kps[g], its input at
// vector g * xs of Xh and its image at vector g * ys of Yh (a stride of 0
// reuses one block).  Chunks of cv vectors (cv divides vpk, so a chunk
// never spans two groups) go through two device slots: the host->device
// copy of chunk i + 1, the apply of chunk i and the device->host copy of
// chunk i - 1 overlap on three streams.
static pcx_status apply_host_pipeline(pcx_ctx* c, const char* who, const pcx::KParams* kps, int nk, int vpk,
                                      const void* Xh, size_t xs, void* Yh, size_t ys, int cv, int precision,
                                      cudaStream_t s) {
  const size_t vbytes = pcx_vector_length(c) * (precision == PCX_FP64 ? 16 : 8);
  const size_t slot = (size_t)cv * vbytes;
  cudaError_t e = cudaSuccess;
  if (2 * slot > c->stage_bytes) {
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(c, who, e);
    if (c->stage_x) cudaFree(c->stage_x);
    if (c->stage_y) cudaFree(c->stage_y);
    c->stage_x = c->stage_y = nullptr;
    c->stage_bytes = 0;
    e = cudaMalloc(&c->stage_x, 2 * slot);
    if (e == cudaSuccess) e = cudaMalloc(&c->stage_y, 2 * slot);
    if (e != cudaSuccess) return cuda_fail(c, who, e);
    c->stage_bytes = 2 * slot;
  }
  for (int i = 0; i < 2 && e == cudaSuccess; ++i)
    if (!c->copy_stream[i]) e = cudaStreamCreateWithFlags(&c->copy_stream[i], cudaStreamNonBlocking);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i)
    for (int j = 0; j < 2 && e == cudaSuccess; ++j)
      if (!c->slot_event[i][j]) e = cudaEventCreateWithFlags(&c->slot_event[i][j], cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(c, who, e);
  cudaStream_t h2d = c->copy_stream[0], d2h = c->copy_stream[1];
  cudaEvent_t* loaded = c->slot_event[0];    // chunk in stage_x[slot]
  cudaEvent_t* applied = c->slot_event[1];   // stage_x[slot] read, stage_y[slot] written
  cudaEvent_t* stored = c->slot_event[2];    // stage_y[slot] copied out
  // earlier work of the caller's stream comes first
  if ((e = cudaEventRecord(applied[0], s)) != cudaSuccess) return cuda_fail(c, who, e);
  if ((e = cudaStreamWaitEvent(h2d, applied[0], 0)) != cudaSuccess) return cuda_fail(c, who, e);
  const int per_group = (vpk + cv - 1) / cv;
  const long long nch = (long long)nk * per_group;
  for (long long ch = 0; ch < nch && e == cudaSuccess; ++ch) {
    const int g = (int)(ch / per_group), j0 = (int)(ch % per_group) * cv;
    const int sl = (int)(ch & 1), nv = vpk - j0 < cv ? vpk - j0 : cv;
    char* sx = static_cast<char*>(c->stage_x) + sl * slot;
    char* sy = static_cast<char*>(c->stage_y) + sl * slot;
    const size_t xoff = ((size_t)g * xs + j0) * vbytes, yoff = ((size_t)g * ys + j0) * vbytes;
    const size_t bytes = (size_t)nv * vbytes;
    if (ch >= 2) e = cudaStreamWaitEvent(h2d, applied[sl], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sx, static_cast<const char*>(Xh) + xoff, bytes, cudaMemcpyHostToDevice, h2d);
    if (e == cudaSuccess) e = cudaEventRecord(loaded[sl], h2d);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, loaded[sl], 0);
    if (e == cudaSuccess && ch >= 2) e = cudaStreamWaitEvent(s, stored[sl], 0);
    if (e == cudaSuccess) e = pcx::launch_apply(c, kps[g], sx, sy, nv, precision, s);
    if (e == cudaSuccess) e = cudaEventRecord(applied[sl], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(d2h, applied[sl], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(static_cast<char*>(Yh) + yoff, sy, bytes, cudaMemcpyDeviceToHost, d2h);
    if (e == cudaSuccess) e = cudaEventRecord(stored[sl], d2h);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(d2h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, who, e);
}

pcx_status pcx_apply_host(pcx_ctx* c, const double k[3], double gamma, const void* Xh, void* Yh, int nvec,
                          int precision, void* stream) {
  pcx_status st = check_block(c, "pcx_apply_host", Xh, Yh, nvec, precision);
  if (st != PCX_OK || nvec == 0) return st;
  if (!k) return inval(c, "pcx_apply_host: NULL k");
  // chunks of about an eighth of the block, at most 4 vectors: only one
  // chunk's copies are exposed
  int cv = (nvec + 7) / 8;
  cv = cv > 4 ? 4 : cv;
  const pcx::KParams kp = pcx::make_kparams(c, k, gamma);
  return apply_host_pipeline(c, "pcx_apply_host", &kp, 1, nvec, Xh, 0, Yh, 0, cv, precision,
                             static_cast<cudaStream_t>(stream));
}

pcx_status pcx_apply_kbatch_host(pcx_ctx* c, const double* kpts, int nk, double gamma, const void* Xh, int x_stride,
                                 void* Yh, int y_stride, int vec_per_k, int precision, void* stream) {
  if (nk < 0 || vec_per_k < 0) return inval(c, "pcx_apply_kbatch_host: nk, vec_per_k must be >= 0");
  if (x_stride < 0 || y_stride < 0) return inval(c, "pcx_apply_kbatch_host: strides must be >= 0");
  if ((long long)nk * vec_per_k > (1LL << 24)) return inval(c, "pcx_apply_kbatch_host: too many vectors");
  pcx_status st = check_block(c, "pcx_apply_kbatch_host", Xh, Yh, nk * vec_per_k, precision);
  if (st != PCX_OK || nk == 0 || vec_per_k == 0) return st;
  if (!kpts) return inval(c, "pcx_apply_kbatch_host: NULL kpts");
  std::vector<pcx::KParams> kps(nk);
  for (int i = 0; i < nk; ++i) kps[i] = pcx::make_kparams(c, kpts + 3 * i, gamma);
  // the largest chunk of at most 4 vectors that divides vec_per_k
  int cv = 1;
  for (int d = 4; d >= 1; --d)
    if (vec_per_k % d == 0) {
      cv = d;
      break;
    }
  return apply_host_pipeline(c, "pcx_apply_kbatch_host", kps.data(), nk, vec_per_k, Xh, (size_t)x_stride, Yh,
                             (size_t)y_stride, cv, precision, static_cast<cudaStream_t>(stream));
}

pcx_status pcx_precond(pcx_ctx* c, const double k[3], double gamma, const void* R, void* W, int nvec, int precision,
                       void* stream) {
  pcx_status st = check_block(c, "pcx_precond", R, W, nvec, precision);
  if (st != PCX_OK || nvec == 0) return st;
  if (!k) return inval(c, "pcx_precond: NULL k");
  const size_t bytes = pcx_vector_length(c) * nvec * (precision == PCX_FP64 ? 16 : 8);
  if (R != W && ranges_overlap(R, bytes, W, bytes)) return inval(c, "pcx_precond: R and W partially overlap");
  pcx::KParams kp = pcx::make_kparams(c, k, gamma);
  cudaError_t e = pcx::launch_precond(c, kp, R, W, nvec, precision, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_precond", e);
}

pcx_status pcx_div_norms(pcx_ctx* c, const double k[3], const void* X, int nvec, int precision, double* out,
                         void* stream) {
  pcx_status st = check_block(c, "pcx_div_norms", X, X, nvec, precision);
  if (st != PCX_OK) return st;
  if (!k || !out) return inval(c, "pcx_div_norms: NULL k or out");
  if (nvec > 65535) return inval(c, "pcx_div_norms: nvec > 65535");
  pcx::KParams kp = pcx::make_kparams(c, k, 0.0);
  cudaError_t e = pcx::launch_div_norms(c, kp, X, nvec, precision, out, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_div_norms", e);
}

pcx_status pcx_apply_kbatch(pcx_ctx* c, const double* kpts, int nk, double gamma, const void* X, void* Y,
                            int vec_per_k, int precision, void* stream) {
  if (nk < 0 || vec_per_k < 0) return inval(c, "pcx_apply_kbatch: nk, vec_per_k must be >= 0");
  if ((long long)nk * vec_per_k > (1LL << 24)) return inval(c, "pcx_apply_kbatch: too many vectors");
  const int nvec = nk * vec_per_k;
  pcx_status st = check_block(c, "pcx_apply_kbatch", X, Y, nvec, precision);
  if (st != PCX_OK || nvec == 0) return st;
  if (!kpts) return inval(c, "pcx_apply_kbatch: NULL kpts");
  const size_t bytes = pcx_vector_length(c) * nvec * (precision == PCX_FP64 ? 16 : 8);
  if (ranges_overlap(X, bytes, Y, bytes)) return inval(c, "pcx_apply_kbatch: X and Y overlap");
  std::vector<pcx::KParams> kps(nk);
  for (int i = 0; i < nk; ++i) kps[i] = pcx::make_kparams(c, kpts + 3 * i, gamma);
  cudaError_t e = pcx::launch_apply_kbatch(c, kps.data(), nk, vec_per_k, X, Y, precision,
                                           static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_apply_kbatch", e);
}

pcx_status pcx_set_apply_graphs(pcx_ctx* c, int enable) {
  if (!c) return inval(nullptr, "pcx_set_apply_graphs: NULL context");
  if (!enable) pcx::free_apply_graphs(c);
  c->use_graphs = enable ? 1 : 0;
  return PCX_OK;
}

pcx_status pcx_set_cnn_form(pcx_ctx* c, int flags) {
  if (!c) return inval(nullptr, "pcx_set_cnn_form: NULL context");
  if (flags & ~(PCX_CNN_HERMITIAN | PCX_CNN_BF16)) return inval(c, "pcx_set_cnn_form: unknown flag");
  c->cnn_form = flags;
  return PCX_OK;
}

pcx_status pcx_set_apply_path(pcx_ctx* c, int path) {
  if (!c) return inval(nullptr, "pcx_set_apply_path: NULL context");
  if (path != PCX_APPLY_AUTO && path != PCX_APPLY_FIVE_PASS && path != PCX_APPLY_THREE_PASS)
    return inval(c, "pcx_set_apply_path: path must be PCX_APPLY_AUTO, PCX_APPLY_FIVE_PASS or PCX_APPLY_THREE_PASS");
  if (path != c->apply_path) pcx::free_apply_graphs(c);   // captured chains hold the old kernels
  c->apply_path = path;
  return PCX_OK;
}

pcx_status pcx_set_apply_variant(pcx_ctx* c, int x_variant, int z_variant) {
  if (!c) return inval(nullptr, "pcx_set_apply_variant: NULL context");
  if (x_variant < -1 || x_variant >= pcx::X3_VARIANTS || z_variant < -1 || z_variant >= pcx::Z3_VARIANTS)
    return inval(c, "pcx_set_apply_variant: x_variant must be in [-1, 2] and z_variant in [-1, 1]");
  if (x_variant != c->x3_variant || z_variant != c->z3_variant) pcx::free_apply_graphs(c);
  c->x3_variant = x_variant;
  c->z3_variant = z_variant;
  return PCX_OK;
}

pcx_status pcx_get_apply_variant(const pcx_ctx* c, int* x_variant, int* z_variant) {
  if (!c) return inval(nullptr, "pcx_get_apply_variant: NULL context");
  if (x_variant) *x_variant = c->x3_variant >= 0 ? c->x3_variant : PCX_X3_VARIANT;
  if (z_variant) *z_variant = c->z3_variant >= 0 ? c->z3_variant : PCX_Z3_VARIANT;
  return PCX_OK;
}

pcx_status pcx_set_penalty_form(pcx_ctx* c, int form) {
  if (!c) return inval(nullptr, "pcx_set_penalty_form: NULL context");
  if (form != PCX_PENALTY_SCALAR && form != PCX_PENALTY_PER_MODE && form != PCX_PENALTY_PROJECTOR)
    return inval(c, "pcx_set_penalty_form: form must be PCX_PENALTY_SCALAR, PCX_PENALTY_PER_MODE or "
                    "PCX_PENALTY_PROJECTOR");
  if (form != c->penalty_form) pcx::free_apply_graphs(c);
  c->penalty_form = form;
  return PCX_OK;
}

int pcx_get_penalty_form(const pcx_ctx* c) { return c ? c->penalty_form : -1; }

int pcx_get_apply_path(const pcx_ctx* c, int precision) {
  if (!c || (precision != PCX_FP64 && precision != PCX_FP32)) return -1;
  return pcx::effective_apply_path(c, precision);
}

pcx_status pcx_autotune(pcx_ctx* c, int precision, int nvec, void* stream, pcx_tune_result* out) {
  if (!c) return inval(nullptr, "pcx_autotune: NULL context");
  if (precision != PCX_FP64 && precision != PCX_FP32) return inval(c, "pcx_autotune: bad precision");
  if (nvec < 1 || nvec > 1024) return inval(c, "pcx_autotune: need 1 <= nvec <= 1024");
  cudaError_t e = pcx::autotune_apply(c, precision, nvec, static_cast<cudaStream_t>(stream), out);
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_autotune", e);
}

pcx_status pcx_sandwich_precond(pcx_ctx* c, const double k[3], double gamma, const void* R, void* W, int nvec,
                                int precision, void* stream) {
  pcx_status st = check_block(c, "pcx_sandwich_precond", R, W, nvec, precision);
  if (st != PCX_OK || nvec == 0) return st;
  if (!k) return inval(c, "pcx_sandwich_precond: NULL k");
  const size_t bytes = pcx_vector_length(c) * nvec * (precision == PCX_FP64 ? 16 : 8);
  if (R != W && ranges_overlap(R, bytes, W, bytes)) return inval(c, "pcx_sandwich_precond: R and W partially overlap");
  pcx::KParams kp = pcx::make_kparams(c, k, gamma);
  cudaError_t e = pcx::sandwich_precond(c, kp, R, W, nvec, precision, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_sandwich_precond", e);
}

static pcx_status check_cnn(pcx_ctx* c, const char* who, int nvec) {
  if (!c) return inval(nullptr, std::string(who) + ": NULL context");
  if (c->n < 8) return inval(c, std::string(who) + ": needs N >= 8");
  if (nvec < 0 || nvec > 32767) return inval(c, std::string(who) + ": need 0 <= nvec <= 32767");
  return PCX_OK;
}

pcx_status pcx_cnn_init(uint64_t seed, float* params, void* stream) {
  if (!params) return inval(nullptr, "pcx_cnn_init: NULL params");
  cudaError_t e = pcx::cnn::init_params(params, seed, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(nullptr, "pcx_cnn_init", e);
}

pcx_status pcx_cnn_gates(pcx_ctx* c, const float* params, float* gates, void* stream) {
  pcx_status st = check_cnn(c, "pcx_cnn_gates", 1);
  if (st != PCX_OK) return st;
  if (!params || !gates || !aligned16(gates)) return inval(c, "pcx_cnn_gates: NULL or misaligned buffer");
  cudaError_t e = pcx::cnn_gates(c, params, gates, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_cnn_gates", e);
}

pcx_status pcx_cnn_forward(pcx_ctx* c, const float* params, const float* gates, const void* U, void* Y, int nvec,
                           void* stream) {
  pcx_status st = check_cnn(c, "pcx_cnn_forward", nvec);
  if (st != PCX_OK || nvec == 0) return st;
  if (!params || !gates || !U || !Y || !aligned16(U) || !aligned16(Y))
    return inval(c, "pcx_cnn_forward: NULL or misaligned buffer");
  const size_t bytes = pcx_vector_length(c) * nvec * 8;
  if (ranges_overlap(U, bytes, Y, bytes)) return inval(c, "pcx_cnn_forward: U and Y overlap");
  cudaError_t e = pcx::cnn_forward(c, params, gates, U, Y, nvec, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_cnn_forward", e);
}

pcx_status pcx_cnn_grad(pcx_ctx* c, const float* params, const void* U, const void* T, const double* w, int nvec,
                        float* grad, int accumulate, double* loss, void* stream) {
  pcx_status st = check_cnn(c, "pcx_cnn_grad", nvec);
  if (st != PCX_OK) return st;
  if (nvec < 1) return inval(c, "pcx_cnn_grad: nvec < 1");
  if (!params || !U || !T || !w || !grad || !aligned16(U) || !aligned16(T))
    return inval(c, "pcx_cnn_grad: NULL or misaligned buffer");
  cudaError_t e = pcx::cnn_grad(c, params, U, T, w, nvec, grad, accumulate ? 1 : 0, loss,
                                static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_cnn_grad", e);
}

pcx_status pcx_cnn_adam(float* params, const float* grad, float* m, float* v, int step, float lr, void* stream) {
  if (!params || !grad || !m || !v || step < 1 || !(lr > 0)) return inval(nullptr, "pcx_cnn_adam: bad argument");
  cudaError_t e = pcx::cnn::adam(params, grad, m, v, pcx::cnn::NPARAMS, step, lr, 0.9f, 0.999f, 1e-8f,
                                 static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(nullptr, "pcx_cnn_adam", e);
}

pcx_status pcx_cnn_precond(pcx_ctx* c, const double k[3], double gamma, const float* params, const float* gates,
                           const void* R, void* W, int nvec, void* stream) {
  pcx_status st = check_cnn(c, "pcx_cnn_precond", nvec);
  if (st != PCX_OK || nvec == 0) return st;
  if (!k || !params || !gates || !R || !W || !aligned16(R) || !aligned16(W))
    return inval(c, "pcx_cnn_precond: NULL or misaligned buffer");
  const size_t bytes = pcx_vector_length(c) * nvec * 8;
  if (R != W && ranges_overlap(R, bytes, W, bytes)) return inval(c, "pcx_cnn_precond: R and W partially overlap");
  pcx::KParams kp = pcx::make_kparams(c, k, gamma);
  cudaError_t e = pcx::cnn_precond(c, kp, params, gates, R, W, nvec, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_cnn_precond", e);
}

pcx_status pcx_cnn_pairs(pcx_ctx* c, const double k[3], double gamma, const void* R, const void* E, void* U, void* T,
                         double* enorm2, int nvec, void* stream) {
  pcx_status st = check_cnn(c, "pcx_cnn_pairs", nvec);
  if (st != PCX_OK || nvec == 0) return st;
  if (!k || !R || !E || !U || !T || !aligned16(R) || !aligned16(E) || !aligned16(U) || !aligned16(T))
    return inval(c, "pcx_cnn_pairs: NULL or misaligned buffer");
  pcx::KParams kp = pcx::make_kparams(c, k, gamma);
  cudaError_t e = pcx::cnn_pairs(c, kp, R, E, U, T, enorm2, nvec, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_cnn_pairs", e);
}

pcx_status pcx_cg_solve(pcx_ctx* c, const double k[3], double gamma, const void* R, void* E, int nvec, double tol,
                        int maxit, int* iters, double* relres, void* stream) {
  pcx_status st = check_cnn(c, "pcx_cg_solve", nvec);
  if (st != PCX_OK || nvec == 0) return st;
  if (!k || !R || !E || !aligned16(R) || !aligned16(E) || !(tol > 0) || maxit < 1)
    return inval(c, "pcx_cg_solve: bad argument");
  pcx::KParams kp = pcx::make_kparams(c, k, gamma);
  cudaError_t e = pcx::cg_solve(c, kp, R, E, nvec, tol, maxit, iters, relres, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_cg_solve", e);
}

pcx_status pcx_set_gram_path(int path) {
  if (path != PCX_GRAM_AUTO && path != PCX_GRAM_TENSOR && path != PCX_GRAM_FP32) return PCX_EINVAL;
  pcx::set_gram_path(path);
  return PCX_OK;
}

int pcx_get_gram_path(void) { return pcx::get_gram_path(); }

pcx_status pcx_gram(pcx_ctx* c, const void* A, int na, const void* B, int nb, size_t L, int precision, void* G,
                    void* stream) {
  if (precision != PCX_FP64 && precision != PCX_FP32) return inval(c, "pcx_gram: bad precision");
  if (na < 1 || nb < 1 || na > 128 || nb > 128) return inval(c, "pcx_gram: need 1 <= na, nb <= 128");
  if (!A || !B || !G || !aligned16(A) || !aligned16(B) || !aligned16(G))
    return inval(c, "pcx_gram: NULL or misaligned buffer");
  cudaError_t e = pcx::launch_gram(A, na, B, nb, L, precision, static_cast<double*>(G), static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_gram", e);
}

pcx_status pcx_gram_mixed(pcx_ctx* c, const void* A, int na, const void* B, int nb, size_t L, void* G, void* stream) {
  if (na < 1 || nb < 1 || na > 128 || nb > 128) return inval(c, "pcx_gram_mixed: need 1 <= na, nb <= 128");
  if (!A || !B || !G || !aligned16(A) || !aligned16(B) || !aligned16(G))
    return inval(c, "pcx_gram_mixed: NULL or misaligned buffer");
  cudaError_t e = pcx::launch_gram_x(A, na, nullptr, 0, B, nb, L, static_cast<double*>(G),
                                     static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_gram_mixed", e);
}

pcx_status pcx_combine(pcx_ctx* c, const void* S, int ns, const void* C, int ny, double beta, void* Y, size_t L,
                       int precision, void* stream) {
  if (precision != PCX_FP64 && precision != PCX_FP32) return inval(c, "pcx_combine: bad precision");
  if (ns < 1 || ny < 1 || ns > 256 || ny > 256) return inval(c, "pcx_combine: need 1 <= ns, ny <= 256");
  if (!S || !C || !Y || !aligned16(S) || !aligned16(Y) || !aligned16(C))
    return inval(c, "pcx_combine: NULL or misaligned buffer");
  const size_t es = precision == PCX_FP64 ? 16 : 8;
  if (ranges_overlap(S, ns * L * es, Y, ny * L * es)) return inval(c, "pcx_combine: S and Y overlap");
  cudaError_t e = pcx::launch_combine(S, ns, static_cast<const double*>(C), ny, beta, Y, L, precision,
                                      static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_combine", e);
}

pcx_status pcx_residual(pcx_ctx* c, const void* X, const void* AX, const double* theta, void* R, double* norms_out,
                        int nvec, size_t L, int precision, void* stream) {
  if (precision != PCX_FP64 && precision != PCX_FP32) return inval(c, "pcx_residual: bad precision");
  if (nvec < 0) return inval(c, "pcx_residual: nvec < 0");
  if (!X || !AX || !theta || !R || !norms_out || !aligned16(X) || !aligned16(AX) || !aligned16(R))
    return inval(c, "pcx_residual: NULL or misaligned buffer");
  cudaError_t e = pcx::launch_residual(X, AX, theta, R, norms_out, nvec, L, precision, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PCX_OK : cuda_fail(c, "pcx_residual", e);
}

pcx_status pcx_rr_eig(int m, const double* ga, const double* gb, double drop_tol, double* theta, double* cvec,
                      int* rank) {
  if (m < 1 || m > 512 || !ga || !gb || !theta || !cvec || !rank) return inval(nullptr, "pcx_rr_eig: bad argument");
  std::vector<pcx::cd> a((size_t)m * m), b((size_t)m * m);
  std::memcpy(a.data(), ga, sizeof(double) * 2 * m * m);
  std::memcpy(b.data(), gb, sizeof(double) * 2 * m * m);
  std::vector<double> th;
  std::vector<pcx::cd> cm;
  const int r = pcx::gen_eig(m, a, b, drop_tol, th, cm);
  *rank = r;
  if (r < 0) {
    g_err = "pcx_rr_eig: metric matrix is not positive definite";
    return PCX_ENUMERIC;
  }
  std::memcpy(theta, th.data(), sizeof(double) * r);
  std::memcpy(cvec, cm.data(), sizeof(double) * 2 * (size_t)m * r);
  return PCX_OK;
}

pcx_status pcx_solve(pcx_ctx* c, const double* kpts, int nk, int nev, double tol, const pcx_solve_opts* opts,
                     double* eig_out, double* res_out, int* iters_out, void* vec_out, void* stream) {
  if (!c) return inval(nullptr, "pcx_solve: NULL context");
  if (vec_out && !aligned16(vec_out)) return inval(c, "pcx_solve: vec_out must be 16-byte aligned");
  try {
    return pcx::solve(c, kpts, nk, nev, tol, opts, eig_out, res_out, iters_out, vec_out,
                      static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    c->err = "pcx_solve: out of host memory";
    return PCX_ENOMEM;
  }
}

}  // extern "C"
