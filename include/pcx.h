/*
 * pcx.h -- C ABI of a GB300 (sm_103a) library for the kernel-compensated
 * Yee-scheme Maxwell eigenproblem of 3D photonic crystals in anisotropic
 * media (arXiv:2511.17107).
 *
 * The discrete problem (Sec. 2.3, eq. kc_formulation): find the smallest
 * positive eigenvalues w_h^2 of
 *
 *     Op = A M A^H + gamma B^H B      on C^{3 N^3},
 *
 * A the Bloch-phased Yee curl (Sec. 2.1 eq. yee_ABmatrix, Sec. 2.2
 * eq. ct_blocks), B the Yee divergence, M the per-cell discrete inverse
 * permittivity M_Trivial (Sec. 3.2.1 eq. trivial_trivial).  The library works
 * in the Fourier basis x = F3^H H (Sec. 2.4 eq. matrixfree_kcform), where
 *
 *     Op_F x = K_A F3^H M F3 K_A^H x + gamma K_B x.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid: N points per axis, N a power of two with 8 <= N <= 256; h = 1/N.
 * Vector block: `nvec` vectors, each 3 N^3 complex numbers laid out
 *   [vec][component 0..2][p3 or z][p2 or y][p1 or x], x fastest, complex
 *   interleaved (re, im).  PCX_FP64 -> double2 (complex128),
 *   PCX_FP32 -> float2 (complex64).  Fourier mode index p_j in [0, N).
 * Device pointers: allocated by the caller (e.g. PyTorch), never freed or
 *   retained by the library; they must be 16-byte aligned.
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Every device entry point only enqueues work on that stream,
 *   except where it says it synchronises.
 * Bloch vector k: Cartesian, 3 doubles (Sec. 1 eq. intro_magneticshifted).
 * gamma: a value <= 0 selects the practical rule of Remark 2.6
 *   (eq. kc_settingofgamma1): 4 pi^2 if k = 0 or |k| >= 1, else 4 pi^2/|k|^2.
 * Errors: every call returns a pcx_status; nothing aborts, nothing traps on
 *   the device.  pcx_last_error() gives a message for the last failing call
 *   on a context.  Invalid arguments never reach a kernel.
 * Threads: a context serves one host thread at a time (its apply scratch,
 *   host staging slots, graph cache, kernel choices and error message are
 *   shared state); use one context per thread for concurrent calls.
 *   pcx_solve's k-points in flight run on threads of its own, each with its
 *   own buffers.
 */
#ifndef PCX_H
#define PCX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pcx_ctx pcx_ctx;

typedef enum {
  PCX_OK = 0,
  PCX_EINVAL = -1,   /* invalid argument (sizes, pointers, alignment)        */
  PCX_ENOMEM = -2,   /* device or host allocation failed                      */
  PCX_ENOTHPD = -3,  /* a cell block of M is not Hermitian positive definite  */
  PCX_ENOCONV = -4,  /* eigensolver hit its iteration cap (partial results)   */
  PCX_ENUMERIC = -5, /* NaN / Inf, or a breakdown the solver cannot repair    */
  PCX_ECUDA = -6     /* a CUDA runtime call failed                            */
} pcx_status;

enum { PCX_FP64 = 0, PCX_FP32 = 1 };

/* Shape kinds of a structure description (Cartesian coordinates, the
 * structure is periodic with the unit cube; see pcx_setup). */
enum {
  PCX_SHAPE_SPHERE = 0,  /* p = cx, cy, cz, r                                  */
  PCX_SHAPE_SEGMENT = 1, /* p = x0, y0, z0, x1, y1, z1, r  (flat-capped rod)   */
  PCX_SHAPE_BOX = 2,     /* p = lox, loy, loz, hix, hiy, hiz  (lo <= x < hi)   */
  PCX_SHAPE_GYROID = 3   /* p = t, mode: g(x) > t (mode 0) or |g(x)| > t (1),
                            g = sin(2pi x)cos(2pi y) + sin(2pi y)cos(2pi z)
                              + sin(2pi z)cos(2pi x)  (Sec. 4)                 */
};

typedef struct {
  int kind;
  int material;   /* index into pcx_setup_desc.eps */
  double p[9];
} pcx_shape;

enum { PCX_CT_SUMMED = 0, PCX_CT_LITERAL = 1 };

typedef struct {
  int n;                 /* grid points per axis (power of two, 8..256)           */
  int stencil_m;         /* 1 = Yee (2nd order) ... 5 (10th order), Sec. 2.5      */
  int ct_reading;        /* PCX_CT_SUMMED (default) or PCX_CT_LITERAL, see below  */
  double lattice[9];     /* row-major 3x3 matrix A whose COLUMNS are a1, a2, a3   */
  int n_mat;             /* number of materials                                   */
  const double* eps;     /* n_mat x 3 x 3 complex PERMITTIVITY, row-major,
                            (re, im) interleaved: 18 doubles per material (host)  */
  int background;        /* material of points outside every shape                */
  int n_shape;
  const pcx_shape* shapes;      /* host; the first shape containing a point wins  */
  const double* cell_blocks;    /* optional host array (NULL = sample shapes):
                            N^3 x 9 already-inverted blocks, cell order z, y, x:
                            d1, d2, d3, re o12, im o12, re o13, im o13, re o23,
                            im o23 (M_k = [[d1,o12,o13],[.,d2,o23],[.,.,d3]],
                            Hermitian)                                           */
  int m_kind;            /* PCX_M_TRIVIAL (0, default) or PCX_M_CROSSDOF, below  */
  int crossdof_unchecked; /* 1: build an M_CrossDoF context even where the
                            sufficient HPD conditions of Sec. 3.3 do not hold
                            (as the paper's ill-conditioned case of Sec. 4.4
                            does); M may then be indefinite.  0 (default):
                            such a context is refused with PCX_ENOTHPD      */
} pcx_setup_desc;

/* m_kind: the discrete inverse permittivity M of the apply (Sec. 3.2).
 * PCX_M_TRIVIAL: eq. trivial_trivial, one 3x3 block per cell (diagonal from
 *   the E1, E2, E3 points, off-diagonals from the volume centre).
 * PCX_M_CROSSDOF: eq. crossdof_herm, the off-diagonal couplings carried
 *   between the staggered E points by symmetrised four-point means,
 *   block (i, j) = (diag(e_ij at E_i) T_ij + T_ij diag(e_ij at E_j)) / 2
 *   with e_ij = (eps^{-1})_ij of the material at each point and T_ij of eq.
 *   crossdof_Tmat read from the componentwise template eq.
 *   crossdof_xytemplate (T_12: mean over x in {i-1, i}, y in {j-1/2,
 *   j+1/2}; T_13, T_23 alike).  It needs a structure sampled from shapes
 *   (not cell_blocks, at most 255 materials).  It is accepted when the
 *   sufficient conditions of Sec. 3.3 hold: every material's epsilon_1 has
 *   eigenvalues in (0, 1], and either one off-diagonal position is zero in
 *   every material or every assembled row is strictly diagonally dominant
 *   (else PCX_ENOTHPD naming the first failing row, unless
 *   crossdof_unchecked is set).  The apply then runs seven passes: the
 *   z-axis sandwich is split into an inverse z transform, a real-space
 *   stencil pass and a forward z transform.  pcx_sandwich_precond keeps
 *   the per-cell M_Trivial inverse (an approximate inverse either way). */
enum { PCX_M_TRIVIAL = 0, PCX_M_CROSSDOF = 1 };

/*
 * pcx_setup -- build a context: sample the structure and assemble M.
 *
 * Sec. 2.1 eqs. yee_edgefacedofs / yee_volumedofs (staggered points, 1-based
 * i,j,k): E1 at ((i-1/2)h, jh, kh), E2 at (ih, (j-1/2)h, kh), E3 at
 * (ih, jh, (k-1/2)h), volume centres at ((i-1/2)h, (j-1/2)h, (k-1/2)h), in
 * fractional coordinates x'; the material is looked up at the physical
 * point A x' (Sec. 2.2 eq. ct_replacement).  Each material's permittivity is
 * inverted in FP64 to epsilon_1 (Sec. 1 eq. intro_permittivity).  Cell block
 * (Sec. 3.1 eq. permittivity_diagonal_case, Sec. 3.2.1 eq. trivial_trivial,
 * Lemma 3.5): d_c = (epsilon_1 at the E_c point)_cc, o_ij = (epsilon_1 at
 * the volume centre)_ij.  Every block is checked to be HPD (3x3 Cholesky).
 *
 * ct_reading: the printed coordinate-transform blocks (Sec. 2.2
 * eq. ct_blocks) sum over j without j appearing.  PCX_CT_SUMMED reads
 * hat D_i = sum_j b_ji (D_{1,j} + i kt_j D_{0,j}), b = A^{-1}, kt = A^T k;
 * PCX_CT_LITERAL reads sum_j b_ji D_{1,j} + i k_i D_{0,i}.  Both equal
 * eq. yee_block for the simple cubic lattice.
 *
 * Ownership: copies everything it needs; desc and its arrays may be freed
 * on return.  The context owns M (FP64 and FP32 copies) and all tables on the
 * current device.  Synchronises the device.
 * Errors: PCX_EINVAL (N not a power of two in [8,256], stencil_m not in
 * [1,5] or N < 2 stencil_m, singular lattice, bad material index, NULL
 * pointers), PCX_ENOTHPD (first failing cell named in pcx_last_error; *out
 * still receives the context so that the message can be read),
 * PCX_ENOMEM, PCX_ECUDA.
 */
pcx_status pcx_setup(const pcx_setup_desc* desc, pcx_ctx** out);

/*
 * pcx_sample_host -- the host half of pcx_setup without a device: samples the
 * structure exactly as pcx_setup does and writes the packed cell blocks
 * (N^3 x 9 doubles, layout of pcx_setup_desc.cell_blocks) and, if ids_out is
 * not NULL, the material index of every sample point (4 x N^3 int32: point
 * sets E1, E2, E3, V, each in cell order z, y, x).  *first_bad receives the
 * first cell (linear index) whose block is not HPD, or -1.  Needs no GPU.
 * Errors: as pcx_setup, except that a non-HPD block is reported through
 * *first_bad, not as an error.
 */
pcx_status pcx_sample_host(const pcx_setup_desc* desc, double* blocks_out, int32_t* ids_out, long long* first_bad);

/* Release a context and its device memory (NULL is ignored). */
void pcx_destroy(pcx_ctx* ctx);

/* Message of the last failing call on ctx ("" if none; ctx may be NULL for
 * errors raised before a context exists). */
const char* pcx_last_error(const pcx_ctx* ctx);

/* Grid size and number of complex entries 3 N^3 of one vector. */
int pcx_grid_n(const pcx_ctx* ctx);
size_t pcx_vector_length(const pcx_ctx* ctx);

/*
 * pcx_cell_blocks -- copy the packed cell blocks of M to a host array of
 * N^3 x 9 doubles (layout of pcx_setup_desc.cell_blocks), and the smallest
 * cell eigenvalue to *lambda_min (may be NULL).  Lemma 3.5: the spectrum of M
 * is the union of the cell-block spectra.
 */
pcx_status pcx_cell_blocks(const pcx_ctx* ctx, double* host_out, double* lambda_min);

/*
 * pcx_symbols -- the per-k tables the kernels use (host output).
 * Lemma 2.1 / Prop. 2.8: Lambda_1(p), Lambda_0(p) are the eigenvalues of the
 * circulant D1, D0 (2m-th order first rows of Sec. 2.5 eq.
 * kc:highord:stencil).  Output (each may be NULL):
 *   s_tab  [3][N] complex (6N doubles): S_j(p) = Lambda_1(p) + i kt_j Lambda_0(p)
 *          (PCX_CT_SUMMED) or Lambda_1(p) (PCX_CT_LITERAL);
 *   q_tab  [3][N] complex: 0 (SUMMED) or i k_i Lambda_0(p) (LITERAL);
 *   b      [9] doubles, b = A^{-1} row-major;
 *   gamma_out: the gamma used (rule above when gamma <= 0).
 * The mode symbol is kappa_i(p) = sum_j b_ji S_j(p_j) + Q_i(p_i).
 */
pcx_status pcx_symbols(const pcx_ctx* ctx, const double k[3], double gamma,
                       double* s_tab, double* q_tab, double* b, double* gamma_out);

/*
 * pcx_set_apply_chunk -- tuning knob of pcx_apply: the number of vectors
 * that run through all five FFT passes before the next ones start (their
 * work space is meant to stay resident in L2).  chunk <= 0 restores the
 * default (largest count whose vectors fill at most half of L2, >= 1).
 * Host-only; affects calls issued afterwards.
 */
pcx_status pcx_set_apply_chunk(pcx_ctx* ctx, int chunk);

/* The chunk pcx_apply uses for `precision` (vectors per five-pass sweep);
 * one call launches 5 * ceil(nvec / chunk) kernels.  0 if ctx is NULL. */
int pcx_get_apply_chunk(const pcx_ctx* ctx, int precision);

/*
 * pcx_apply -- Y = Op_F X for a block of nvec vectors (device, stream-ordered).
 *
 * Sec. 2.4 eq. matrixfree_kcform with Prop. 2.8:
 *   u = K_A^H x = -conj(kappa) x x            (per mode)
 *   e = F3 u,  m = M e (per cell, Sec. 3.2.1),  w = F3^H m
 *   y = K_A w + gamma K_B x = kappa x w + gamma conj(kappa) (kappa . x)
 * with F3 = F (x) F (x) F, F_ij = w^{(i-1)(j-1)}/sqrt(N), w = exp(2 pi i/N)
 * (Lemma 2.1).  X and Y: nvec vectors in `precision`; X and Y must not
 * overlap.  Y is the work space of the transforms; the context owns a
 * scratch array of chunk x N^3 complex entries (gamma kappa . x carried from
 * the first pass to the last), allocated on first use and grown on demand
 * (the growth synchronises the device).
 * Errors: PCX_EINVAL (NULL or misaligned pointers, nvec < 0, X == Y,
 * bad precision), PCX_ECUDA (launch failure).  nvec == 0 is a no-op.
 */
pcx_status pcx_apply(pcx_ctx* ctx, const double k[3], double gamma, const void* X, void* Y,
                     int nvec, int precision, void* stream);

/*
 * pcx_apply_noalloc -- pcx_apply for callers that cannot allocate device
 * memory.  The paper has no counterpart: this entry point exists for
 * integration, not for the method.  Some callers must not call cudaMalloc or
 * cudaFree during their steady state: an application whose device memory is
 * carved out up front by its own pool or framework allocator and must not be
 * fragmented or oversubscribed by a library, or a real-time loop where an
 * allocation's latency (and its implicit device synchronisation) is not
 * acceptable.
 * pcx_apply may allocate (its scratch grows on demand); this variant never
 * does: no cudaMalloc, no cudaFree, no allocating library routine.
 *
 * Its scratch (gamma kappa . x for one chunk of vectors, and for M_CrossDoF
 * also the real-space field of its stencil pass) lives in a file-scope
 * device array of PCX_NOALLOC_SCRATCH_BYTES (32 MiB) that every GPU loading
 * the library holds until the process exits.  Limit: one vector's scratch
 * must fit: N^3 complex entries (M_Trivial), 4 N^3 (M_CrossDoF), i.e.
 * entries * 8 bytes (PCX_FP32) or * 16 bytes (PCX_FP64) <= 32 MiB -- every
 * N <= 128 in both precisions for M_Trivial, N <= 64 for M_CrossDoF; larger
 * grids are rejected with PCX_EINVAL before any launch.  Vectors are
 * processed in chunks that fit the array.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  The address is kept
 * for the life of the
 * process: a cudaDeviceReset while the library is loaded is not supported.
 * The context's device must be current (PCX_EINVAL otherwise).
 * The array is shared by every call and keeps the last call's contents;
 * nothing in it needs to start at zero (the first FFT pass writes all of it
 * before the last pass reads it).  Calls whose execution overlaps on the GPU
 * (other streams, other threads) race on the array: serialise them.
 * Arguments, results and errors otherwise as pcx_apply.
 */
#define PCX_NOALLOC_SCRATCH_BYTES (32u << 20)
pcx_status pcx_apply_noalloc(pcx_ctx* ctx, const double k[3], double gamma, const void* X, void* Y, int nvec,
                             int precision, void* stream);

/*
 * pcx_apply_kbatch -- Y = Op(k_i) X for nk Bloch vectors at once: X and Y hold
 * nk groups of vec_per_k vectors ([nk][vec_per_k][3][N^3], group i at
 * kpts[3 i .. 3 i + 2], HOST doubles), gamma as in pcx_apply (<= 0: the rule
 * per k).  One launch per pass sweeps every (k, vector) pair, each x pass
 * reading its k from a device table (the y and z passes do not depend on
 * k).  Same results as nk calls of pcx_apply.  The table lives in the
 * context: concurrent calls on one context must share one stream.
 */
pcx_status pcx_apply_kbatch(pcx_ctx* ctx, const double* kpts, int nk, double gamma, const void* X, void* Y,
                            int vec_per_k, int precision, void* stream);

/*
 * pcx_set_apply_graphs -- enable (1) or disable (0) CUDA-graph replay of the
 * apply launch chain in pcx_apply and pcx_solve: a (buffers, size, k, stream)
 * combination runs eagerly the first time, is captured the second time and
 * replayed afterwards (up to 64 graphs per context).  Needs a non-default
 * stream; on the legacy default stream the apply stays eager.  Disabling
 * frees the cached graphs.
 */
pcx_status pcx_set_apply_graphs(pcx_ctx* ctx, int enable);

/*
 * pcx_set_apply_path -- pass structure of the apply (and of the T0
 * preconditioner, which runs on the same chain) in this context:
 *   PCX_APPLY_FIVE_PASS   five HBM round trips per vector: one batch of 1D
 *                         transforms per axis x, y, z (the z pass carrying the
 *                         M sandwich), then y, x;
 *   PCX_APPLY_THREE_PASS  three round trips: the y transforms split four-step
 *                         (N = RA RB) and folded into the x and z passes,
 *                         the intermediates kept in place in Y; complex64 at
 *                         N = 32, 64, 128 (elsewhere the five-pass chain runs);
 *   PCX_APPLY_AUTO        (default) the three-pass form where it exists.
 * Both compute the same operator (Sec. 2.4 eq. matrixfree_kcform); the
 * rounding differs.  M_CrossDoF contexts always use their seven-pass chain.
 * PCX_EINVAL for another value.
 */
#define PCX_APPLY_AUTO 0
#define PCX_APPLY_FIVE_PASS 1
#define PCX_APPLY_THREE_PASS 2
pcx_status pcx_set_apply_path(pcx_ctx* ctx, int path);
/* The pass structure the apply of this context runs at `precision`:
 * PCX_APPLY_FIVE_PASS or PCX_APPLY_THREE_PASS (7 for the seven-pass
 * M_CrossDoF chain); -1 for a NULL context or a bad precision. */
int pcx_get_apply_path(const pcx_ctx* ctx, int precision);

/*
 * pcx_set_penalty_form -- how the penalty term of this context weighs the
 * Fourier modes (every later apply, preconditioner and solve uses it):
 *   PCX_PENALTY_SCALAR    (default) one coefficient gamma for all modes,
 *                         gamma K_B (Sec. 2.3, eq. kc_formulation); gamma <= 0
 *                         in a call selects the rule of Remark 2.6.
 *   PCX_PENALTY_PER_MODE  mode p carries gamma_p = gamma max(1, 1/|kappa_p|^2),
 *                         and gamma <= 0 in a call selects gamma = 4 pi^2:
 *                         the rule of Remark 2.6 applied per mode with the
 *                         mode's own B eigenvalue |kappa_p|^2 (Lemma
 *                         kc_ABblock) in place of |k|^2.
 * Both leave the divergence-free eigenpairs unchanged: the penalty acts only
 * on span(conj kappa_p) per mode, where Op reduces to gamma_p |kappa_p|^2,
 * so with the per-mode rule every spurious eigenvalue is at least 4 pi^2
 * (the condition gamma lambda^B >= lambda_m^A of Prop. 2.5 holds mode by
 * mode, also for k outside the first zone).  What changes is the top of the
 * spectrum: the scalar rule puts it at about 12 N^2 4 pi^2 / |k|^2 for
 * 0 < |k| < 1, the per-mode rule at 12 N^2 4 pi^2 whatever k, which bounds
 * the FP64 rounding floor of the residual (about 1e-16 times the largest
 * eigenvalue) below 1e-8 at N = 128 near Gamma.
 *   PCX_PENALTY_PROJECTOR gamma_p = gamma / |kappa_p|^2 (gamma <= 0 in a call:
 *                         16 pi^2, four times the rule's value, since all
 *                         N^3 penalty eigenvalues sit at gamma and a cluster
 *                         just above the wanted ones would slow LOBPCG or
 *                         enter the wanted set): gamma_p K_B(p) is gamma times the
 *                         projector onto conj(kappa_p), every penalty
 *                         eigenvalue equals gamma, and the top of the
 *                         spectrum is that of A M A^H (about 12 N^2 / eps_min)
 *                         instead of 12 N^2 4 pi^2 -- a lower FP32 rounding
 *                         floor for the mixed scheme.  Prop. 2.5's condition
 *                         needs gamma >= lambda_m^A, as with the rule.
 * Switching the form frees the captured apply graphs.  PCX_EINVAL for
 * another value.
 */
#define PCX_PENALTY_SCALAR 0
#define PCX_PENALTY_PER_MODE 1
#define PCX_PENALTY_PROJECTOR 2
pcx_status pcx_set_penalty_form(pcx_ctx* ctx, int form);
/* The penalty form of this context; -1 for a NULL context. */
int pcx_get_penalty_form(const pcx_ctx* ctx);

/*
 * pcx_set_apply_variant -- kernel variants of the three-pass chain in this
 * context (the arithmetic, and so every result, is the same; only the
 * schedule differs):
 *   x_variant (passes A and C): 0 -- one row's global loads at a time, three
 *     CTAs per SM; 1 -- three rows' loads issued together, three CTAs per
 *     SM; 2 -- six rows' loads together, two CTAs per SM; 3 -- pass A as
 *     a persistent kernel, two CTAs per SM, that copies the next tile's
 *     input rows into shared memory asynchronously (cp.async) while it
 *     transforms the current tile, pass C as in 1 (input vectors not
 *     16-byte aligned run variant 1);
 *   z_variant (pass B): 0 -- one z tile per CTA; 1 -- a persistent
 *     warp-specialised kernel, one CTA per SM, in which half the warps
 *     transform one tile buffer while the other half store the previous
 *     tile and load the next one into the second buffer.
 * -1 selects the build's default (x 3, z 0).  pcx_autotune sets both.
 * Changing them frees the captured apply graphs.  PCX_EINVAL out of range.
 */
pcx_status pcx_set_apply_variant(pcx_ctx* ctx, int x_variant, int z_variant);
/* The variants in effect (defaults resolved); either pointer may be NULL. */
pcx_status pcx_get_apply_variant(const pcx_ctx* ctx, int* x_variant, int* z_variant);

/* Result of pcx_autotune. */
typedef struct {
  int chunk;            /* vectors per launch chunk chosen                         */
  int graphs;           /* 1 if graph replay was faster and is enabled            */
  double us_per_vector; /* measured time of the chosen configuration              */
  int candidates;       /* configurations timed (0 when from a cache)             */
  int from_cache;       /* 0 measured, 1 process cache, 2 the PCX_TUNE_CACHE file  */
  int path;             /* pass structure chosen: PCX_APPLY_FIVE_PASS or
                           PCX_APPLY_THREE_PASS                                    */
  int x_variant;        /* three-pass kernel variants chosen (pcx_set_apply_variant; */
  int z_variant;        /* -1 when the five-pass chain was chosen)                   */
} pcx_tune_result;

/*
 * pcx_autotune -- choose the apply launch configuration of this context for
 * blocks of nvec vectors at `precision`: for each pass structure the
 * context has (the five-pass chain, and the three-pass one where it
 * exists; see pcx_set_apply_path), every chunk size 1, 2, 4, ... <=
 * min(nvec, 64) (and nvec) is timed with CUDA events on `stream` (two warm
 * and three timed applies on random vectors); when the three-pass chain
 * wins, every pair of its kernel variants (pcx_set_apply_variant) at the
 * best chunk; then graph replay of the best configuration when `stream` is
 * not the default stream.  The choice is applied to the context (as
 * pcx_set_apply_path / pcx_set_apply_chunk / pcx_set_apply_variant /
 * pcx_set_apply_graphs would) and cached
 * per device, SM count, N, precision and nvec for the process; when the
 * environment variable PCX_TUNE_CACHE names a file, results are read from and
 * appended to it.  Allocates two blocks of nvec vectors while timing;
 * synchronises `stream`.  *out (optional) receives the result.
 */
pcx_status pcx_autotune(pcx_ctx* ctx, int precision, int nvec, void* stream, pcx_tune_result* out);

/*
 * pcx_apply_host -- pcx_apply on HOST buffers, synchronising `stream` before
 * returning.  The block moves in chunks (an eighth of it, at most 4 vectors)
 * through two device staging slots: the host->device copy of one chunk, the
 * apply of the previous one (on `stream`) and the device->host copy of the
 * one before run at the same time, the copies on two streams of the
 * context.  Pinned host memory gives the overlap and full copy bandwidth;
 * pageable memory also works.  Staging buffers, streams and events are
 * owned by the context.
 */
pcx_status pcx_apply_host(pcx_ctx* ctx, const double k[3], double gamma, const void* X_host,
                          void* Y_host, int nvec, int precision, void* stream);

/*
 * pcx_apply_kbatch_host -- pcx_apply_kbatch on HOST buffers: for each of the
 * nk Bloch vectors kpts[3 i .. 3 i + 2] (i < nk), the vec_per_k vectors
 * starting at vector i * x_stride of X_host are applied with k_i and their
 * images written at vector i * y_stride of Y_host (strides in vectors; 0
 * reuses one block for every k, a later k's images overwriting an
 * earlier's).  One pipeline for the whole batch, as in pcx_apply_host: chunks
 * of up to 4 vectors that divide vec_per_k, host->device copy, apply and
 * device->host copy of consecutive chunks overlapping on three streams, so
 * the pipeline fills and drains once per call rather than once per k.
 * Synchronises `stream` before returning.  PCX_EINVAL for negative counts or
 * strides, more than 2^24 vectors, NULL or misaligned buffers.
 */
pcx_status pcx_apply_kbatch_host(pcx_ctx* ctx, const double* kpts, int nk, double gamma, const void* X_host,
                                 int x_stride, void* Y_host, int y_stride, int vec_per_k, int precision,
                                 void* stream);

/*
 * pcx_precond -- W = K_P^{-1} R per Fourier mode (device, stream-ordered).
 * Sec. 2.4 eqs. matrixfree_diagP / matrixfree_finalform:
 *   K_P = K_A K_A^H + gamma K_B = |kappa|^2 I + (gamma - 1) conj(kappa) kappa^T,
 *   K_P^{-1} = I/|kappa|^2 + (1/gamma - 1) conj(kappa) kappa^T / |kappa|^4
 * (Sherman-Morrison).  A mode with kappa = 0 (only k = 0, p = 0: the null
 * space H of Prop. 2.5) maps to 0.  R == W (in place) is allowed.
 */
pcx_status pcx_precond(pcx_ctx* ctx, const double k[3], double gamma, const void* R, void* W,
                       int nvec, int precision, void* stream);

/*
 * pcx_gram -- G = A^H B for two blocks of columns of length L (complex):
 * G[i*nb + j] = sum_l conj(A_i[l]) B_j[l], written as na x nb complex128
 * (interleaved doubles) to the DEVICE buffer G.  The Gram products of the
 * Rayleigh-Ritz step (Sec. 4: LOBPCG).  Column i of A starts at
 * A + i * L elements.  precision PCX_FP32: FP32 products accumulated per
 * chunk of rows and summed in FP64, on the path pcx_set_gram_path selects:
 * the tensor cores (tcgen05 TF32 with hi/lo error compensation) or the
 * FP32 pipes (register-blocked FMAs, double-float sums across chunks), for
 * na, nb <= 64, even L and 16-byte aligned A, B; a generic CUDA-core
 * kernel otherwise.  PCX_FP64: double-float products and sums on the FP32
 * pipes (error-free product and sum transformations, about 2^-44 relative
 * per term) with the per-block partials summed in FP64.  1 <= na, nb <= 128.
 */
pcx_status pcx_gram(pcx_ctx* ctx, const void* A, int na, const void* B, int nb, size_t L,
                    int precision, void* G, void* stream);

/*
 * pcx_set_gram_path -- process-wide choice of the complex64 Gram kernel
 * (pcx_gram and every Gram product inside pcx_solve): PCX_GRAM_AUTO (the
 * default choice for the shape), PCX_GRAM_TENSOR (tcgen05 TF32 hi/lo) or
 * PCX_GRAM_FP32 (FP32 pipes).  Both paths agree to FP32 accuracy; the
 * choice changes speed only.  Returns PCX_EINVAL for another value.
 * pcx_get_gram_path returns the current choice.
 */
#define PCX_GRAM_AUTO 0
#define PCX_GRAM_TENSOR 1
#define PCX_GRAM_FP32 2
pcx_status pcx_set_gram_path(int path);
int pcx_get_gram_path(void);

/*
 * pcx_gram_mixed -- G = A^H B with A complex128 (na columns) and B complex64
 * (nb columns), both of length L, written as na x nb complex128 to the
 * DEVICE buffer G (G[i*nb + j], interleaved doubles).  The X rows of the
 * Rayleigh-Ritz matrices in the mixed-precision refinement (Sec. 4: LOBPCG
 * with the block X held in FP64 and the search directions in FP32).
 * Accuracy: about 2^-44 relative to ||A_i|| ||B_j|| (double-float sums on
 * the FP32 pipes).  Entries of A must lie inside the FP32 range: magnitudes
 * below 2^-126 count as 0, magnitudes at or above 2^128 give NaN.  A, B, G
 * 16-byte aligned device pointers; 1 <= na, nb <= 128.  Uses a per-device
 * scratch buffer owned by the library: concurrent calls on different streams
 * of one device must be serialised by the caller.
 */
pcx_status pcx_gram_mixed(pcx_ctx* ctx, const void* A, int na, const void* B, int nb, size_t L, void* G,
                          void* stream);

/*
 * pcx_combine -- Y_j = sum_i S_i C[i*ny + j]  (+ beta * Y_j if beta != 0):
 * tall x small product of the Rayleigh-Ritz update (Sec. 4: LOBPCG).
 * S: ns columns of length L; C: DEVICE ns x ny complex128; Y: ny columns;
 * Y must not overlap S.  1 <= ns <= 256, 1 <= ny <= 256.
 */
pcx_status pcx_combine(pcx_ctx* ctx, const void* S, int ns, const void* C, int ny, double beta,
                       void* Y, size_t L, int precision, void* stream);

/*
 * pcx_residual -- R_j = AX_j - theta_j X_j and the squared norms
 * out[j] = ||R_j||^2, out[nvec + j] = ||X_j||^2 (DEVICE doubles), giving
 * Res_j = ||R_j|| / ||X_j|| of Sec. 4 eq. exp_relativeresidual.  theta:
 * DEVICE doubles.  R may alias AX.
 */
pcx_status pcx_residual(pcx_ctx* ctx, const void* X, const void* AX, const double* theta, void* R,
                        double* norms_out, int nvec, size_t L, int precision, void* stream);

/*
 * pcx_rr_eig -- the small generalised Hermitian eigenproblem of the
 * Rayleigh-Ritz step (Sec. 4: LOBPCG), on the HOST in FP64:
 *   G_A c = theta G_B c,  G_A, G_B m x m Hermitian (row-major complex128,
 *   interleaved doubles), G_B positive semi-definite.
 * Directions in which the diagonally scaled G_B has an eigenvalue
 * <= drop_tol * (its largest) are discarded (rank-revealing orthonormalisation
 * of the search space); *rank receives the number r kept.  theta[r] ascending;
 * cvec: m x r row-major complex128 with G_B-orthonormal columns.  Buffers must
 * hold m values / m*m complex entries.  Errors: PCX_EINVAL (m outside
 * [1, 512], NULL), PCX_ENUMERIC (G_B has a non-positive diagonal entry).
 * Needs no GPU.
 */
pcx_status pcx_rr_eig(int m, const double* ga, const double* gb, double drop_tol, double* theta, double* cvec,
                      int* rank);

/*
 * pcx_div_norms -- per column of X (Fourier basis, nvec vectors):
 *   out[j] = x_j^H K_B x_j = sum over modes |kappa(p) . x_j(p)|^2,
 *   out[nvec + j] = ||x_j||^2   (DEVICE doubles).
 * K_B = [K_1^H; K_2^H; K_3^H][K_1 K_2 K_3] is the Fourier form of B^H B
 * (Prop. 2.8), so out[j] = ||B h_j||^2 for the real-space field h_j = F3_3 x_j:
 * the penalty share of a Rayleigh quotient is gamma out[j] / (theta out[nvec+j]).
 * Under PCX_PENALTY_PER_MODE or _PROJECTOR each mode's term is weighted by gamma_p / gamma,
 * so out[j] = x_j^H (sum_p gamma_p K_B(p)) x_j / gamma and the share formula
 * stands.
 * Stream-ordered; X as in pcx_apply.
 */
pcx_status pcx_div_norms(pcx_ctx* ctx, const double k[3], const void* X, int nvec, int precision, double* out,
                         void* stream);

/*
 * pcx_sandwich_precond -- W = T0 R, the curl-sandwich approximate inverse of
 * the compensated operator (Johnson and Joannopoulos, Opt. Express 8 (2001)
 * 173, restated with the symbols of Prop. 2.8; not in the paper):
 *   T0 r = K_A F3_3^H eps F3_3 (K_A^H r / |k|^2) / |k|^2 + K_B r / (gamma |k|^4)
 * with eps = M^{-1} cell by cell and |k|^2 = sum_i |kappa_i|^2 per mode (a
 * mode with |k| = 0 maps to 0).  Exact inverse for a homogeneous isotropic
 * medium (K_A K_A^H + K_B = |k|^2 I); K_P^{-1} is T0 with eps = I.  Runs
 * on the five fused passes of the apply (eps = adj(M) / det(M) in the
 * middle pass), so it costs one apply.  Device buffers as in pcx_apply;
 * W may alias R.
 */
pcx_status pcx_sandwich_precond(pcx_ctx* ctx, const double k[3], double gamma, const void* R, void* W, int nvec,
                                int precision, void* stream);

/* ---------------------------------------------------------------------------
 * Learned correction of the preconditioner (the paper has no learned part):
 *
 *   T(r) = T0 r + K_A F3_3^H g(e) / |k|^2,   e = F3_3 (K_A^H r / |k|^2),
 *
 * T0 as in pcx_sandwich_precond, F3_3 the unitary 3D DFT of each component
 * (Sec. 2.4: x = F3_3^H H), and g a three-layer circular 3D convolution net
 * (3x3x3 taps) acting next to eps on the real-space field e, with the same
 * weights on its real and imaginary parts:
 *   g1 = sigmoid(conv(f, V1) + c1),  g2 = sigmoid(conv(f, V2) + c2)
 *   y  = conv(g2 * conv(g1 * conv(u, W1), W2), W3)
 * where f are the 9 reals of the cell blocks of M (Sec. 3.2.1: d1, d2, d3,
 * Re/Im M12, M13, M23).  g is linear in u, so T is a complex-linear map.
 * conv(x, w)[o][z][y][x] = sum_{i,dz,dy,dx} w[o][i][t] x[i][z+dz][y+dy][x+dx]
 * with tap t = (dz+1)*9 + (dy+1)*3 + (dx+1) and periodic wrap-around.
 * Parameters: one DEVICE float array of PCX_CNN_NPARAMS entries laid out as
 * W1[8][3][27], W2[8][8][27], W3[3][8][27], V1[8][9][27], c1[8],
 * V2[8][9][27], c2[8].  Fields are complex64 [nvec][3][N][N][N], grid sizes
 * 8 <= N (powers of two), FP32 arithmetic.  Device pointers, stream-ordered;
 * workspace is owned by the context and grows on demand.
 * ------------------------------------------------------------------------- */
#define PCX_CNN_HIDDEN 8
#define PCX_CNN_NPARAMS (PCX_CNN_HIDDEN * 3 * 27 + PCX_CNN_HIDDEN * PCX_CNN_HIDDEN * 27 + 3 * PCX_CNN_HIDDEN * 27 + \
                         2 * (PCX_CNN_HIDDEN * 9 * 27 + PCX_CNN_HIDDEN))

/* Form of the correction in this context (flags; default 0: g in FP32):
 *   PCX_CNN_HERMITIAN  g_s = (g + g^T) / 2 in place of g, with the transpose
 *                      g^T(u) = conv^T(g1 * conv^T(g2 * conv^T(u, W3), W2), W1)
 *                      (conv^T the adjoint of conv): a symmetric real map,
 *                      so T = T0 + B^H g_s B (B = F3_3 K_A^H / |k|^2) is
 *                      Hermitian like T0;
 *   PCX_CNN_BF16       every convolution uses its weights rounded to BF16
 *                      (round to nearest even), accumulating in FP32; the
 *                      parameters themselves stay FP32 (the master copy that
 *                      pcx_cnn_adam updates), and pcx_cnn_grad returns the
 *                      gradient of the rounded network (straight through).
 * Applies to pcx_cnn_forward, pcx_cnn_grad, pcx_cnn_precond and the learned
 * path of pcx_solve.  PCX_EINVAL for other bits. */
#define PCX_CNN_HERMITIAN 1
#define PCX_CNN_BF16 2
pcx_status pcx_set_cnn_form(pcx_ctx* ctx, int flags);

/* Random initial parameters (seeded): W1, W2, V1, V2 normal with variance
 * 1/fan-in, W3 = 0 and c = 0 (so T starts as K_P^{-1}). */
pcx_status pcx_cnn_init(uint64_t seed, float* params, void* stream);

/* The two gate fields g1, g2 of this context's structure: gates = DEVICE
 * 2 * 8 * N^3 floats, g1 then g2, each [8][N^3]. */
pcx_status pcx_cnn_gates(pcx_ctx* ctx, const float* params, float* gates, void* stream);

/* Y = g(Re U) + i g(Im U) for nvec real-space fields U (Y may not alias U). */
pcx_status pcx_cnn_forward(pcx_ctx* ctx, const float* params, const float* gates, const void* U, void* Y, int nvec,
                           void* stream);

/* Loss L = sum_v w[v] ||g(U_v) - T_v||^2 (w: HOST doubles, nvec) and its
 * gradient with respect to every parameter, written (accumulate = 0) or
 * added (accumulate = 1) to the DEVICE float array grad (PCX_CNN_NPARAMS).
 * *loss (HOST) receives L; synchronises `stream` when loss is not NULL. */
pcx_status pcx_cnn_grad(pcx_ctx* ctx, const float* params, const void* U, const void* T, const double* w, int nvec,
                        float* grad, int accumulate, double* loss, void* stream);

/* One Adam step (Kingma and Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8) on
 * DEVICE arrays of PCX_CNN_NPARAMS floats; step counts from 1. */
pcx_status pcx_cnn_adam(float* params, const float* grad, float* m, float* v, int step, float lr, void* stream);

/* W = T(R) for nvec Fourier-basis vectors (complex64), gates from
 * pcx_cnn_gates.  gamma <= 0: the rule of Remark 2.6.  W may alias R. */
pcx_status pcx_cnn_precond(pcx_ctx* ctx, const double k[3], double gamma, const float* params, const float* gates,
                           const void* R, void* W, int nvec, void* stream);

/* Training pairs from residuals R and targets E = Op^{-1} R (Fourier basis,
 * complex64): the net's input U = F3_3 (K_A^H R / |k|^2) and target
 * T = F3_3 K_A^H (E - T0 R) (real space; g(U) = T makes T(R) = E), and
 * enorm2[v] = ||K_A^H E_v||^2 (HOST doubles; synchronises when not NULL). */
pcx_status pcx_cnn_pairs(pcx_ctx* ctx, const double k[3], double gamma, const void* R, const void* E, void* U,
                         void* T, double* enorm2, int nvec, void* stream);

/* E = Op^{-1} R for nvec complex64 vectors by preconditioned conjugate
 * gradients (K_P^{-1}; FP32 vectors, FP64 scalars), one recursion per column,
 * until every ||R - Op E|| / ||R|| <= tol or maxit iterations.  *iters and
 * relres[nvec] (HOST, optional) report the iterations and the recursion's
 * relative residuals.  At k = 0 the p = 0 mode of R must be zero (Prop. 2.5). */
pcx_status pcx_cg_solve(pcx_ctx* ctx, const double k[3], double gamma, const void* R, void* E, int nvec, double tol,
                        int maxit, int* iters, double* relres, void* stream);

/* Counters and wall-clock split of one pcx_solve call (summed over k).
 * Phase times are measured with a stream synchronisation after each phase
 * when this struct is requested, so they add up to the total. */
typedef struct {
  int iters_fp32;        /* LOBPCG iterations with FP32 storage and apply          */
  int iters_fp64;        /* LOBPCG iterations with FP64 storage and apply          */
  long long applies_fp32;  /* vectors applied in FP32                                */
  long long applies_fp64;  /* vectors applied in FP64                                */
  double ms_total;
  double ms_apply;       /* pcx_apply work                                          */
  double ms_gram;        /* Gram products (device) and their transfer to the host  */
  double ms_rr;          /* host Rayleigh-Ritz and Cholesky                         */
  double ms_other;       /* preconditioner, combinations, residuals, conversions   */
  int gamma_raises;      /* times the spurious-mode guard raised gamma (all k)     */
  double gamma_last;     /* penalty coefficient used at the last k                 */
  double ms_precond;     /* preconditioner (K_P^{-1} or the learned T)              */
  int learned_fallbacks; /* k-points at which the learned correction fell back     */
  int dumped;            /* residual columns written to dump_R                      */
  int history_len;       /* entries written to opts.res_history                     */
} pcx_solve_stats;

/* Eigensolver options (pcx_solve).  Zero-initialised fields take defaults. */
typedef struct {
  int block;          /* vectors per block (>= nev; default nev + 4)               */
  int maxit;          /* iteration cap per k (default 1000)                        */
  int precision;      /* PCX_FP64: all FP64.  PCX_FP32: mixed -- FP32 apply and
                         storage, FP64 Rayleigh-Ritz, then FP64 refinement         */
  double switch_tol;  /* mixed: switch to FP64 when all Res_j <= this (default 1e-4) */
  uint64_t seed;      /* initial block seed (default 20251117)                     */
  int verbose;        /* print per-iteration residuals to stderr                   */
  pcx_solve_stats* stats;  /* optional output (host), zeroed and filled by pcx_solve */
  double gamma;       /* penalty coefficient; 0: the rule of Sec. 2 per k
                         (4 pi^2 if k = 0 or |k| >= 1, else 4 pi^2 / |k|^2)        */
  double penalty_tol; /* spurious-mode guard: after convergence, a wanted pair
                         with gamma x^H K_B x / (theta ||x||^2) above this is a
                         penalty mode (Prop. 2.3: eigenvalue gamma * lambda^B);
                         gamma is then multiplied by 4 and k re-solved, at most
                         4 times (then PCX_ENUMERIC).  0: default 1e-6;
                         negative: guard off                                      */
  const float* cnn_params; /* DEVICE parameters of the learned correction
                         (PCX_CNN_NPARAMS floats) or NULL.  With PCX_FP32 the
                         search directions use T(R) (pcx_cnn_precond) until the
                         worst wanted residual has not dropped for 3
                         iterations at a k; then the precond_kind one         */
  void* dump_R;       /* optional DEVICE complex64 buffer of dump_cap vectors:
                         the FP32 phase copies its active residual columns
                         every dump_every iterations until it is full
                         (training data for the learned correction)           */
  int dump_cap;
  int dump_every;     /* 0: every iteration                                    */
  int precond_kind;   /* 0: K_P^{-1} (eq. matrixfree_finalform, default);
                         1: the curl-sandwich T0 (pcx_sandwich_precond)        */
  int learned_patience; /* iterations without a 10% drop of the worst
                         residual below its best before the learned
                         correction falls back to the base preconditioner
                         (0: 3; negative: never)                               */
  double fp32_floor;  /* mixed: the FP32 phase also ends once the worst wanted
                         residual is <= fp32_floor * 2^-24 * theta_top, with
                         theta_top the largest Ritz value of the search space
                         (FP32 rounding of Op x, of size 2^-24 ||Op|| ||x||,
                         bounds the residual that phase can reach; at 128^3
                         the FP32 phase stalls near 1000 * 2^-24 * theta_top).
                         0: default 1024; negative: off                       */
  const void* x0;     /* optional DEVICE initial block, block vectors in the FP64
                         layout ([block][3 N^3] complex128), used at every k in
                         place of the seeded random block (a warm start, e.g.
                         the previous k's eigenvectors along a band path); the
                         p = 0 mode is deflated from it at k = 0.  NaN/Inf or a
                         rank-deficient block gives PCX_ENUMERIC.  NULL: random */
  int k_concurrency;  /* k-points solved at the same time (0 or 1: one after the
                         other).  Each k in flight gets its own host thread,
                         stream, search-space buffers and apply scratch (13
                         block x 3 N^3 complex entries in the working
                         precision, plus 5 block x 3 N^3 complex128 for the
                         FP64 refinement of PCX_FP32: 10.5 + 8 GB at 128^3,
                         block 16), so the GPU
                         runs one k's kernels while another k's host does its
                         Rayleigh-Ritz step.  Same results as one after the
                         other.  Not with cnn_params or dump_R (they share the
                         context's workspace): those solve one k at a time.  */
  double* res_history;  /* optional HOST array: the worst wanted residual
                         max_{j < nev} Res_j after every LOBPCG iteration (FP32
                         phase and refinement, in the order they run), at most
                         res_history_cap entries; stats->history_len gives the
                         count.  With k-points in flight their entries
                         interleave.                                          */
  int res_history_cap;
} pcx_solve_opts;

/*
 * pcx_solve -- smallest nev positive eigenvalues w_h^2 at each of nk Bloch
 * vectors (host kpts, nk x 3), by block LOBPCG with soft locking (Sec. 4;
 * Knyazev 2001) preconditioned by K_P^{-1}: Rayleigh-Ritz on span{X, W, P},
 * W = K_P^{-1} R, converged columns keep their place in X but get no new W
 * or P.  Converged when every Res_j <= tol (eq. exp_relativeresidual).  At
 * k = 0 the p = 0 mode of every block is deflated (Prop. 2.5: null space H).
 * Outputs (host, any may be NULL): eig_out[nk*nev] ascending per k,
 * res_out[nk*nev], iters_out[nk].  vec_out: optional DEVICE buffer for the
 * eigenvectors (nk*nev vectors, FP64 layout).  Synchronises `stream`.
 * Errors: PCX_ENOCONV (cap reached; outputs hold the last iterate),
 * PCX_ENUMERIC (NaN/Inf or unrecoverable breakdown), PCX_EINVAL, PCX_ENOMEM,
 * PCX_ECUDA.
 */
pcx_status pcx_solve(pcx_ctx* ctx, const double* kpts, int nk, int nev, double tol,
                     const pcx_solve_opts* opts, double* eig_out, double* res_out,
                     int* iters_out, void* vec_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PCX_H */
