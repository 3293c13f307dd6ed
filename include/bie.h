/*
 * bie.h -- C ABI of the B300 library for the FFT-accelerated surface boundary
 * integral equation method for 3D Helmholtz scattering (singularity swapping
 * for the theta-Fourier coefficients of the single- and double-layer kernels,
 * panel-based generalized Gaussian quadrature, dense solve, field evaluation).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Complex numbers are interleaved double pairs (re, im) ("double2").
 *  - Every array argument marked [dev] is a CUDA device pointer owned by the
 *    caller; [host] pointers are host memory owned by the caller.  The library
 *    never frees caller memory.  Opaque handles (bie_ctx, bie_surface,
 *    bie_matrix) are owned by the library and released by their *_free call.
 *  - All GPU work is enqueued on the stream given to bie_ctx_create and is
 *    asynchronous unless stated otherwise; results are visible after a stream
 *    synchronisation.
 *  - Errors are reported by the return value (bie_status); bie_last_error()
 *    returns a thread-local description of the last failure.  No entry point
 *    aborts, traps or falls back to the CPU: there is no CPU path.
 *  - A context (bie_ctx) owns the pair pipeline's work buffers (grown on
 *    demand, freed by bie_ctx_free); calls on one context are ordered by its
 *    stream, and calls on different contexts (other streams, other host
 *    threads) may run concurrently.  The recurrence coefficient table is one
 *    read-only array per device, allocated on first use and kept until exit.
 *    Every call that launches work checks that the context's device is the
 *    current device (BIE_EINVAL otherwise).
 *  - Index of an unknown / collocation node: (panel*16 + node)*Mth + l, with
 *    panel = 0..Np-1 (uniform panels of [0, L]), node = 0..15 (Gauss-Legendre),
 *    l = 0..Mth-1 (theta_l = 2 pi l / Mth).  The unknown is the weighted
 *    density phi~ = phi J (Section 3, Eq. (S:para)).
 */
#ifndef BIE_H
#define BIE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BIE_OK = 0,
  BIE_EINVAL = 1,        /* invalid argument (null pointer, size out of range) */
  BIE_ENOMEM = 2,        /* device allocation failed */
  BIE_ECUDA = 3,         /* a CUDA call failed; see bie_last_error() */
  BIE_ENOCONV = 4,       /* the solver did not reach the tolerance within maxit */
  BIE_ENAN = 5,          /* NaN/Inf detected in inputs or iterates */
  BIE_ETIMEOUT = 6,      /* a bounded device wait expired */
  BIE_EUNSUPPORTED = 7   /* valid request that this build does not implement */
} bie_status;

typedef struct bie_ctx_s* bie_ctx;
typedef struct bie_surface_s* bie_surface;
typedef struct bie_matrix_s* bie_matrix;
typedef struct bie_batch_s* bie_batch;

/* ---- kernels and operators ------------------------------------------------ */
#define BIE_KERNEL_S 1u  /* e^{ik rho}/rho                      (Section 3, Eq. (Sphi:appr2)) */
#define BIE_KERNEL_K 2u  /* alpha tau1 - tau3 - i beta tau0      (Section 4, Eq. (dis:K))      */
#define BIE_KERNEL_KP 4u /* the same with tau0 = nu(x).(x - y), the target's normal
                            (Section 4, the integrand of the adjoint double layer K')        */

typedef enum {
  BIE_OP_S = 0,          /* S                      (Eq. (bie:S))                          */
  BIE_OP_K = 1,          /* K                                                             */
  BIE_OP_K_PLUS_I = 2,   /* K + I  exterior Dirichlet, double layer (Eq. (bie:Kie))        */
  BIE_OP_K_MINUS_I = 3,  /* K - I  interior Dirichlet, double layer (Eq. (bie:Kie))        */
  BIE_OP_CFIE = 4,       /* I + K - i eta S: exterior Dirichlet, combined field           */
  BIE_OP_KP = 5,         /* K' (adjoint double layer)                                     */
  BIE_OP_KP_PLUS_I = 6,  /* K' + I  interior Neumann (Eq. (bie:Kpie))                      */
  BIE_OP_KP_MINUS_I = 7  /* K' - I  exterior Neumann (Eq. (bie:Kpie))                      */
} bie_operator;

/* ---- context ----------------------------------------------------------------
 * bie_ctx_create: bind a context to the current CUDA device and to cuda_stream
 * (a cudaStream_t; NULL = legacy default stream).  *out receives the handle.
 * Errors: BIE_EINVAL (out == NULL), BIE_ECUDA.                                */
bie_status bie_ctx_create(bie_ctx* out, void* cuda_stream);
void bie_ctx_free(bie_ctx ctx);
const char* bie_last_error(void);
/* Options of a context.  BIE_OPT_FP64_TRANSFORMS (value 0 or 1, default 0): the
 * single layer's transforms, upsampling, products and unpacking in FP64 instead of
 * double-word FP32 arithmetic (about 48 significant bits; both stay within the
 * 1e-12 per-pair bound), in bie_kernel_modes and the assembly calls; a measure of
 * what the narrower arithmetic buys.  The batch scheduler, the allocation-free
 * entry and the double layer's fused kernel are not affected.
 * Errors: BIE_EINVAL.                                                          */
#define BIE_OPT_FP64_TRANSFORMS 1
bie_status bie_ctx_set_option(bie_ctx ctx, int option, int value);

/* Launch trace (measurement): with enable != 0 the context records CUDA events on
 * its stream around every launch of the pair kernels (root, transform, fused),
 * the near fill (one mark per panel group) and the far fill.
 * bie_ctx_trace_read synchronises the stream and returns, per family (0 pair
 * root, 1 pair transform, 2 fused pair kernel, 3 near fill, 4 far fill), the
 * summed event time in ms and the number of marks, then clears the trace.
 * [host] ms double[5], launches int[5].  Errors: BIE_EINVAL, BIE_ECUDA.        */
bie_status bie_ctx_trace(bie_ctx ctx, int enable);
bie_status bie_ctx_trace_read(bie_ctx ctx, double* ms, int* launches);
/* Wait for all work of the context's stream; returns BIE_ECUDA on a device error,
 * BIE_EINVAL if a kernel met an invalid pair, BIE_ETIMEOUT if a bounded device
 * wait expired (both flags are cleared by the call). */
bie_status bie_ctx_sync(bie_ctx ctx);

/* ---- surfaces (Section 2, Eq. (para); Section 3.1) -------------------------
 * kind 0, ellipsoid:  r = (a sin t cos th, b sin t sin th, c cos t), t in [0, pi]
 *                     (axes = a, b, c)
 * kind 1, star:       r = h(t,th) (sin t cos th, sin t sin th, cos t),
 *                     h = 1 + sum_i c_i sin^p_i t cos^q_i t T_i(m_i th),
 *                     T = cos (s_i = 0) or sin (s_i = 1); terms[5*i..5*i+4] =
 *                     (c, p, q, m, s) as doubles, n_terms <= BIE_MAX_TERMS.
 * kind 2, bean (Section 5, Example 2, given there implicitly; parameterised
 *                     by z = cos t and the angle th around each horizontal
 *                     ellipse): r = (sqrt(A) sin t cos th, -0.3 u + sqrt(B) sin t
 *                     sin th, cos t), u = cos(pi cos t), A = 0.64 (1 - 0.1 u),
 *                     B = 0.64 (1 - 0.4 u); no parameters.
 * kind 3, torus (Section 5, Example 3): r = (a w cos t, b w sin t, c sin th),
 *                     w = R + cos th + eps cos(m t), t in [0, 2 pi] periodic;
 *                     axes = (a, b, c), one term (R, eps, m, -, -).
 * kind 4, Fourier torus (Section 5, Example 4): r = (w cos t, w sin t, zeta),
 *                     w = R + sum c_i cos(m_i th + n_i t), zeta = sum c_i
 *                     sin(m_i th + n_i t), t periodic; axes[0] = R, terms
 *                     (c, m, n, -, -).
 * On the tori (kinds 3, 4) the first and last panels are neighbours (Section
 * 3.1, Remark): every panel has two near neighbours, and n_panels >= 3.      */
#define BIE_MAX_TERMS 96
typedef struct {
  int kind;
  int n_terms;
  double axes[3];
  const double* terms;   /* [host] 5*n_terms doubles, ignored for kind 0 */
} bie_surface_desc;

/* 16-node generalized Gaussian rules on the reference panel [-1, 1]
 * (Section 3.1: self and adjacent panels, nodes and weights depend on the
 * target node l).  x[d][l][g], w[d][l][g], d = delta + 1 with delta = -1
 * (source panel left of the target panel), 0 (self), +1 (right).  The panel
 * nodes t_i^l, the far-panel rule and the line-integral rule of the Section 4
 * Remark all use gl_x/gl_w, so results depend only on these tables.         */
typedef struct {
  double x[3][16][16];
  double w[3][16][16];
  double gl_x[16];       /* 16-point Gauss-Legendre nodes on [-1, 1], ascending */
  double gl_w[16];       /* and weights (Section 3.1: t_i^l and Eq. (S1))      */
} bie_quad_tables;

/* bie_surface_sample: sample the surface on the collocation grid (Np panels x
 * 16 Legendre nodes x Mth angles) and on every GGQ source ring (one ring per
 * target node, near panel and GGQ node, Mth angles each): positions, unit
 * normals, Jacobians and the data the pair pipeline needs (Section 2 and the
 * Section 4 Remark on second derivatives).  Allocates device memory owned by
 * the returned handle.  Np in [2, 4096]; Mth even, in [8, 1024], of the form
 * 2^a 3^b 5^c.  Errors: BIE_EINVAL, BIE_ENAN (a NaN or Inf in the descriptor or
 * the tables), BIE_ENOMEM, BIE_ECUDA.                                       */
bie_status bie_surface_sample(bie_ctx ctx, const bie_surface_desc* desc, int n_panels,
                              int m_theta, const bie_quad_tables* ggq, bie_surface* out);
void bie_surface_free(bie_surface s);
/* Number of unknowns N = 16*Np*Mth, and number of near pairs 256*Mth*(3Np-2)
 * (3Np on a torus): targets x GGQ source nodes on the self and adjacent panels. */
int64_t bie_surface_unknowns(bie_surface s);
int64_t bie_surface_near_pairs(bie_surface s);
/* [dev] views owned by the surface: node positions [N][3], unit normals [N][3],
 * Jacobians [N] (double). */
const double* bie_surface_points(bie_surface s);
const double* bie_surface_normals(bie_surface s);
const double* bie_surface_jacobians(bie_surface s);

/* ---- kernel modes (Sections 3.2-3.3, 4) -----------------------------------
 * For each pair p = (target row, source) with target row = flat node index
 * (t_j^l, theta_i) and source = d*16 + g (the GGQ node g of the near panel
 * j + d - 1, cyclic on a torus), write the theta_s-Fourier modes K_m,
 * m = -M..M (M = Mth/2), of each requested kernel (bit mask of
 * BIE_KERNEL_S, _K, _KP; any non-empty subset), computed by singularity
 * swapping: complex root of rho^2 by Newton, smooth factor F = (s_{a,b}/rho^2)^{1/2}
 * (Lemma "singular1"), A_m(b) by the difference recurrence or Miller's
 * recurrence (Eqs. (Am), (diff-recurrence)), zero-padded FFT convolution
 * (Eq. (convolution)), tau_3 by Eqs. (tau3-standard)/(tau3-modified).
 *   pair_row  [dev] int64[n_pairs], pair_src [dev] int32[n_pairs]
 *   modes_out [dev] double2[n_pairs][n_kernels][Mth+1], kernels in bit order
 *   k > 0 wavenumber.
 * Errors: BIE_EINVAL (bad sizes/pointers; a pair whose source panel does not
 * exist yields zeros and BIE_EINVAL after the next bie_ctx_sync), BIE_ECUDA.
 * Not for stream capture: the call may grow its device buffers (cudaMalloc,
 * with a stream synchronisation) and sets the kernels' shared-memory launch
 * attribute for this surface's Mth.  Capture bie_batch_run instead.           */
bie_status bie_kernel_modes(bie_ctx ctx, bie_surface s, unsigned kernels, double k,
                            const int64_t* pair_row, const int32_t* pair_src, int64_t n_pairs,
                            double* modes_out);

/* bie_kernel_modes_noalloc: the same computation as bie_kernel_modes, for
 * callers that must not allocate device memory -- for example code running
 * while another allocator holds the whole device (a framework's caching
 * allocator), or a latency-critical path where cudaMalloc's implicit device
 * synchronisation is not acceptable.  The paper has no counterpart; this is a
 * property of the library.  bie_kernel_modes grows a device work buffer (the
 * per-warp A_m / D_m tables of the recurrences) with cudaMalloc on demand;
 * this entry point uses a fixed array in the library's device image instead
 * (16.8 MB, held on every device that loads the library until the process
 * exits) and calls no cudaMalloc, cudaFree or allocating routine.
 *   Limit: Mth <= 128 (BIE_EINVAL with a message otherwise); any n_pairs (a
 *   fixed grid of 32 CTAs loops over them, so it is slower than
 *   bie_kernel_modes on large inputs).
 *   The first call on a device takes the device addresses of the arrays and
 *   copies the recurrence coefficients into them (cudaGetSymbolAddress,
 *   cudaMemcpyToSymbol) with that device current; make that first call before
 *   any stream capture.  Every call checks that the context's device is the
 *   current device (BIE_EINVAL otherwise), since the addresses are per device.
 *   All calls share the arrays: calls that may overlap on the GPU (other
 *   streams, other host threads) race and must be serialised by the caller.
 *   Nothing in the arrays needs clearing between calls: every table entry is
 *   written before it is read within a call.
 * Arguments, layouts and other errors as bie_kernel_modes.                     */
bie_status bie_kernel_modes_noalloc(bie_ctx ctx, bie_surface s, unsigned kernels, double k,
                                    const int64_t* pair_row, const int32_t* pair_src, int64_t n_pairs,
                                    double* modes_out);

/* Flag for bie_assemble's op and bie_field_eval's rep: the unknown is the
 * density itself (psi), not the weighted density psi J.  Matrix columns are
 * multiplied by the Jacobian of the source node, so the identity of K +- I and
 * of the combined-field operator is I instead of diag(1/J); this second-kind
 * form is much better conditioned for iterative solvers.                      */
#define BIE_UNWEIGHTED 0x100

/* ---- the O(M) route (Section 3.3, "An O(M) approach") ---------------------
 * bie_rho_inv_modes: for each query q with target x = r(t[q], theta[q]) and
 * source ring t_s = ts[q] (t != t_s), the theta_s-Fourier modes
 *   <rho^{-1}>_l = (1/2pi) int_0^{2pi} e^{-i l theta_s} / |r(t_s, theta_s) - x| dtheta_s,
 * l = 0..lmax (<rho^{-1}>_{-l} is the conjugate), by the difference equation of
 * Eq. (lin:diff): the modes of rho^2 from 64 samples, m0 by Eq. (crt:M0) (every
 * mode beyond m0 below eps0 times the largest), the first and last m0 modes by
 * Gauss-Legendre quadrature on panels graded towards the minimiser of rho^2
 * (Eq. (offline:terms)), the others from the banded system Eq. (Axb) by
 * Gaussian elimination with partial pivoting inside the band.
 *   t, theta, ts [dev] double[n]; modes_out [dev] double2[n][lmax + 1];
 *   m0_out [dev] int32[n] or NULL: the m0 of each query.
 *   lmax >= 4d + 1 and <= 65536, where d is the surface's theta-degree (1 for
 *   the ellipsoid, bean and tori, 1 + max m for a star, max m for a Fourier
 *   torus); 2d <= 15.  eps0 in (0, 1e-6]; the paper's value is 1e-14; m0 <= 2d.
 * Accuracy: the route takes rho^2 through its modes, whose rounding (relative
 * to max rho^2) is amplified near the minimiser by 1/min rho^2: it serves
 * pairs that are not extremely close (the paper recommends singularity
 * swapping, bie_kernel_modes, for close pairs unless Mth is very large).
 * Errors: BIE_EINVAL, BIE_ECUDA; a query with t == t_s, a non-finite input or a
 * zero pivot gets NaN modes, and the next bie_ctx_sync returns BIE_ENAN.
 * Not for stream capture (the call may grow its device scratch).              */
bie_status bie_rho_inv_modes(bie_ctx ctx, bie_surface s, const double* t, const double* theta,
                             const double* ts, int64_t n, int lmax, double eps0, double* modes_out,
                             int32_t* m0_out);
/* bie_kernel_modes_banded: single-layer modes K_m, m = -M..M (M = Mth/2), of
 * the pairs of bie_kernel_modes (same pair_row / pair_src encoding and output
 * layout double2[n_pairs][Mth + 1]) through the O(M) route: Eq. (Sphi:appr2)
 * with M0 = M, K_m = sum_j <cos k rho>_j <rho^{-1}>_{m-j} + i <sin(k rho)/rho>_m,
 * the grid modes of cos(k rho) and sin(k rho)/rho (j = -M..M, the Nyquist mode
 * split evenly) from one FFT of length Mth, <rho^{-1}>_l (l <= Mth) as in
 * bie_rho_inv_modes.  Mth <= 1024 and Mth >= 4d + 1.
 * Errors: as bie_rho_inv_modes; invalid pairs as bie_kernel_modes.            */
bie_status bie_kernel_modes_banded(bie_ctx ctx, bie_surface s, double k, const int64_t* pair_row,
                                   const int32_t* pair_src, int64_t n_pairs, double eps0,
                                   double* modes_out);

/* ---- batch scheduler -------------------------------------------------------
 * Many surfaces of uneven size (panels, Mth, wavenumber) in a few launches.
 * bie_batch_create builds a device-resident plan: the near pairs of every
 * surface (all 16*Np*48*Mth enumerated (node, delta, g, theta) pairs, invalid
 * edge pairs give zero weights) are cut into items and grouped by grid size
 * Mth into classes, largest first, so that each class runs at the shared-
 * memory carve and occupancy of its own Mth.
 *  - Single layer alone (kernels = BIE_KERNEL_S): each class runs in chunks
 *    through the root and transform kernels of bie_kernel_modes (per-pair
 *    records in a plan-owned buffer of up to 2^20 pairs at the largest Mth);
 *    the autotuner times chunks of 2^18, 2^19 and 2^20 pairs.
 *  - With a double layer (K or KP): one persistent launch of the fused kernel
 *    per class, resident warps claiming the class's items from an atomic
 *    counter; the autotuner times item sizes {256, 1024, 4096} on a prefix.
 * bie_batch_run resets the counters and launches the classes in order
 * (bie_batch_launches kernels).  It allocates nothing and can be captured in a
 * CUDA graph (call it once before capture).  At most 64 distinct Mth per plan.
 * Output: the Parseval weights of pair p of surface i (its enumerated index)
 * go to row (bie_batch_offset(plan, i) + p) % slot_pairs of weights_out [dev]
 * (the offsets follow the processing order: classes by decreasing Mth,
 * surfaces in their order within a class)
 * double2[nk][slot_pairs][max Mth] (row length = largest Mth of the batch;
 * kernel blocks in bit order).  slot_pairs >= bie_batch_pairs(plan) keeps
 * every row; smaller values make a bounded ring (throughput runs).
 * The surfaces and weights_out must outlive the plan.
 * Errors: BIE_EINVAL, BIE_ENOMEM, BIE_ECUDA, BIE_EUNSUPPORTED.                 */
bie_status bie_batch_create(bie_ctx ctx, int n_surf, const bie_surface* surfs, const double* ks,
                            unsigned kernels, double* weights_out, int64_t slot_pairs, bie_batch* out);
bie_status bie_batch_run(bie_batch plan);
/* bie_batch_set_fill: throughput mode with the GGQ fill (Section 3.4, Eq. (S123)):
 * once every pair of a target panel has its Parseval weights, bie_batch_run
 * folds them with the panel's GGQ / Lagrange coefficients into that panel's
 * near band, as bie_assemble_near_band does for one surface (single layer,
 * weighted density, S scaled by h/2; rows [16 Mth][3][16 Mth], slots of source
 * panels outside the surface zeroed).  Panel f of the run (in processing order)
 * goes to slot f % band_slots of band_ring [dev] double2[band_slots][16 maxMth]
 * [3][16 maxMth] (a bounded per-wave buffer: slots are overwritten), with row
 * length 3*16*Mth of its own surface.  Single-layer plans only.  The ring of
 * weight rows must hold one panel plus one chunk of the plan: the chunk is cut
 * to fit.  band_ring = NULL turns the fill off.
 * Errors: BIE_EINVAL (slot_pairs below a panel plus one item), BIE_EUNSUPPORTED
 * (a plan with a double layer).                                             */
bie_status bie_batch_set_fill(bie_batch plan, double* band_ring, int band_slots);
int64_t bie_batch_pairs(bie_batch plan);
int64_t bie_batch_offset(bie_batch plan, int i);
void bie_batch_config(bie_batch plan, int* item_pairs, int* warps_per_block, int* blocks);
int bie_batch_launches(bie_batch plan);

/* bie_shard_surfaces: split n independent surfaces over world ranks (one GPU
 * each) for batches that do not fit one GPU.  Surfaces share no pairs, so each
 * rank makes a plan of its own surfaces and no data moves between ranks.
 * Greedy longest-processing-time order: owner[i] in [0, world) for cost[i] >= 0
 * (e.g. near pairs times log Mth), load[r] (may be NULL) the summed cost of rank
 * r.  Host only: no device call.  Errors: BIE_EINVAL.                         */
bie_status bie_shard_surfaces(int n, const double* cost, int world, int* owner, double* load);
void bie_batch_free(bie_batch plan);

/* ---- assembly (Section 3.4, Eq. (S1), Section 4) --------------------------
 * Fill the dense N x N matrix of operator op acting on the weighted density:
 * preparation stage (Gauss-Legendre x trapezoid for every block) and
 * correction stage (near blocks |i-j| <= 1, cyclically on a torus, from the
 * pair pipeline, Parseval weights, GGQ weights and Lagrange interpolation to
 * the 16 Legendre nodes).  op: a bie_operator, optionally | BIE_UNWEIGHTED.
 *   A_out [dev] double2[N][N] row-major (row = target), overwritten.
 *   eta   coupling of BIE_OP_CFIE (ignored otherwise).
 * Errors: BIE_EINVAL, BIE_ECUDA.                                              */
bie_status bie_assemble(bie_ctx ctx, bie_surface s, int op, double k, double eta, double* A_out);

/* Correction stage only (the paper's dominant cost, Section 3.4): add
 * (ws_re + i ws_im) times the near-block entries of S and (wk_re + i wk_im)
 * times those of the double layer, K or K' (kernels = BIE_KERNEL_S with at
 * most one of BIE_KERNEL_K, BIE_KERNEL_KP) to A_out [dev]
 * double2[N][N] (row = target).  Entries outside the near blocks are not
 * touched.  Uses a device work buffer of 16*48*Mth*Mth double2 (freed on
 * return, stream-ordered).  Errors: BIE_EINVAL, BIE_ENOMEM, BIE_ECUDA.       */
bie_status bie_assemble_near(bie_ctx ctx, bie_surface s, unsigned kernels, double k,
                             double ws_re, double ws_im, double wk_re, double wk_im, double* A_out);

/* Correction stage into the near band alone (Section 3.4): the same entries
 * as bie_assemble_near adds to a zero matrix, in the band layout
 *   band_out double2[N][3][16*Mth]:  row = target node index,
 *   slot d = (source panel) - (target panel) + 1, entry = column within that
 *   source panel (Legendre node n, theta index) = n*Mth + theta.
 * Slots of source panels outside the surface (d = 0 on the first panel,
 * d = 2 on the last) are zero.  Every entry is overwritten.
 * band_out is either device memory (written in place) or page-locked host
 * memory (cudaHostAlloc / cudaHostRegister): then the band is filled on the
 * device a group of target panels at a time in two staging slots
 * (2 * group * 16*Mth rows, freed on return, stream-ordered) and each group is
 * copied to the host on a second stream while the next group's pair kernels
 * run.  Asynchronous on the ctx stream either way: the band is complete once
 * the ctx stream passes this call (bie_ctx_sync).  Pageable host memory is
 * refused (BIE_EINVAL).  The caller keeps the buffer alive until then.
 * Errors: BIE_EINVAL, BIE_ENOMEM, BIE_ECUDA.  Not for stream capture (as
 * bie_kernel_modes; it also creates a stream and events for the host copies). */
bie_status bie_assemble_near_band(bie_ctx ctx, bie_surface s, unsigned kernels, double k,
                                  double ws_re, double ws_im, double wk_re, double wk_im,
                                  double* band_out);

/* ---- block-diagonal preconditioner ------------------------------------------
 * LU factors, with partial pivoting, of the n / block diagonal blocks
 * A[b block : (b+1) block, same] of the system matrix.  With block = 16 Mth
 * a block is one panel's self interaction (16 Gauss-Legendre rings x Mth
 * samples, every self-panel GGQ correction of Section 3.4).  Factors are FP32
 * complex (an approximate inverse; FGMRES keeps the outer residual in FP64).
 *   A [dev] double2[n][n] row-major (read once; not kept).
 *   32 <= block <= 4096, block divides n.  Holds n * block float2 of device
 *   memory until bie_blockdiag_free.  Synchronises the ctx stream.
 * bie_blockdiag_apply: z = B^{-1} r for nv vectors, r, z [dev] double2[nv][n],
 *   z must not alias r; asynchronous on the ctx stream.
 * Errors: BIE_EINVAL, BIE_ENOMEM, BIE_ECUDA, BIE_ENAN (a block has a zero
 * pivot column; the message names the block).                               */
typedef struct bie_blockdiag_s* bie_blockdiag;
bie_status bie_blockdiag_create(bie_ctx ctx, int64_t n, const double* A, int block, bie_blockdiag* out);
bie_status bie_blockdiag_apply(bie_blockdiag P, const double* r, int nv, double* z);
int64_t bie_blockdiag_size(bie_blockdiag P);
void bie_blockdiag_free(bie_blockdiag P);

/* ---- learned preconditioner ---------------------------------------------------
 * A 4-layer convolutional network on the (t, theta) grid of the unknowns
 * (t = panel * 16 + node rows, Mth columns): 3x3 convolutions
 * 4 -> 32 -> 32 -> 32 -> 2, dilations 1, 2, 4, 1, ReLU after the first three,
 * theta periodic, t zero-padded.  For a residual r its input features are
 * Re r / s, Im r / s, J / mean(J), k / 25 with s = rms(r); the preconditioner
 * is z = B^{-1} r + s (o_0 + i o_1) (B^{-1}: the block-diagonal factors, or 0).
 * Parameters: float[BIE_NET_PARAMS], per layer W[cout][cin][3][3] then
 * bias[cout].  The FP32 master copy is trained (Adam); every pass uses its
 * BF16 rounding with FP32 accumulation.
 * Feature / output tensors: [dev] float[B][C][nt][mt], C = 4 in, 2 out.
 *
 * bie_net_create: params [host] (NULL: seeded He-uniform hidden layers, zero
 *   output layer, zero biases, so that z = B^{-1} r at start).
 * bie_net_forward: y = net(x).
 * bie_net_backward: gradients of sum(gy * net(x)) w.r.t. the parameters
 *   (gparams [dev] float[BIE_NET_PARAMS]) and x (gx, may be NULL).
 * bie_train_set_create: a training system: the surface (grid, J), k, the
 *   system matrix A [dev] double2[N][N] (an FP32 copy is kept, 8 N^2 bytes)
 *   and the block preconditioner used as the base (may be NULL).
 * bie_net_loss_grad: L = (1/nv) sum_v ||A z_v - r_v||^2 / ||r_v||^2 for
 *   r [dev] float2[nv][N] (nv <= 16) and its parameter gradient (gparams
 *   [dev], may be NULL); loss [host].
 * bie_net_train: opts->steps Adam steps; step i uses set i mod n_sets and a
 *   batch of residuals drawn from splitmix64 (seed, step): half complex
 *   white noise, half A x with white x.  loss_history [host] float[steps]
 *   (may be NULL).  Synchronises the ctx stream.
 * bie_net_precond_apply: z = B^{-1} v + s net(features(v)) for nv <= 16
 *   vectors v, z [dev] double2[nv][N] of the surface (block may be NULL).
 * Errors: BIE_EINVAL, BIE_ENOMEM, BIE_ECUDA.                                  */
#define BIE_NET_PARAMS 20258
typedef struct bie_net_s* bie_net;
typedef struct bie_train_set_s* bie_train_set;
typedef struct {
  int steps;
  int batch;         /* 2 .. 16 */
  float lr;
  float beta1, beta2, eps;
  uint64_t seed;
} bie_train_opts;
bie_status bie_net_create(bie_ctx ctx, const float* params, uint64_t seed, bie_net* out);
bie_status bie_net_get_params(bie_net net, float* params);
void bie_net_free(bie_net net);
bie_status bie_net_forward(bie_net net, int B, int nt, int mt, const float* x, float* y);
bie_status bie_net_backward(bie_net net, int B, int nt, int mt, const float* x, const float* gy,
                            float* gparams, float* gx);
bie_status bie_train_set_create(bie_ctx ctx, bie_surface s, double k, const double* A,
                                bie_blockdiag block, bie_train_set* out);
void bie_train_set_free(bie_train_set ts);
bie_status bie_net_loss_grad(bie_net net, bie_train_set ts, const float* r, int nv, float* gparams,
                             float* loss);
bie_status bie_net_train(bie_net net, const bie_train_set* sets, int n_sets, const bie_train_opts* opts,
                         float* loss_history);
bie_status bie_net_precond_apply(bie_net net, bie_blockdiag block, bie_surface s, double k,
                                 const double* v, int nv, double* z);

/* ---- dense solve -------------------------------------------------------------
 * The paper states the system (Section 3.4) and no solver; this one is restarted
 * FGMRES (right preconditioned, classical Gram-Schmidt with re-orthogonalisation)
 * run for up to 16 right-hand sides in lockstep: every iteration makes one pass
 * over the matrix for all of them (a block product), until
 * ||b - A x|| <= tol ||b|| for each.
 *
 * bie_matrix: an assembled system matrix and the low-precision copies the mixed
 * solves read.  The FP64 matrix A [dev] double2[n][n] (row-major) stays
 * caller-owned and must outlive the handle; store (bit mask) adds copies owned by
 * the handle: BIE_STORE_FP32 (FP32 complex, 8 n^2 bytes) and BIE_STORE_BF16X2
 * (split BF16: hi = bf16(a), lo = bf16(a - hi) for every real component, 8 n^2
 * bytes plus padding of rows to 128 and columns to 32, laid out in the tensor
 * cores' shared-memory image).  Made once per matrix, it serves any number of
 * solves.  Asynchronous on the ctx stream.  Errors: BIE_EINVAL, BIE_ENOMEM,
 * BIE_ECUDA.
 * bie_matrix_matvec: y [nr][n] = A x [nr][n] (both [dev] double2, 1 <= nr <= 16)
 * with the product prec: 0 FP64 arithmetic; 1 the FP32 copy (FP32 products,
 * chunk sums in FP64); 2 the split-BF16 copy on the tensor cores (tcgen05,
 * FP32 accumulation, accumulators added in FP64; relative error about 1e-5);
 * 3 FP64 storage with double-word products (about 2^-44; the refinement
 * residual of the mixed solves).  Errors: BIE_EINVAL (a copy the product needs
 * is missing), BIE_ECUDA; a bounded wait that expired inside the tensor-core
 * product is reported by the next bie_solve as BIE_ETIMEOUT.                    */
#define BIE_STORE_FP32 1u
#define BIE_STORE_BF16X2 2u
bie_status bie_matrix_create(bie_ctx ctx, int64_t n, const double* A, unsigned store, bie_matrix* out);
void bie_matrix_free(bie_matrix M);
int64_t bie_matrix_size(bie_matrix M);
bie_status bie_matrix_matvec(bie_matrix M, int prec, const double* x, int nr, double* y);

/* bie_solve_matrix: solve A x = b for nrhs right-hand sides (blocks of up to 16).
 *   rhs [dev] double2[nrhs][n];  x [dev] double2[nrhs][n] (initial guess in,
 *   solution out).
 *   prec 0 = FP64 products throughout; 1 = FP32 products inside FGMRES, 2 =
 *        split-BF16 tensor-core products inside FGMRES, each with FP64-accurate
 *        iterative refinement outside (residuals b - A x by product 3, x += dx);
 *        prec 1 and 2 need the matching copy in the bie_matrix.
 *   precond 0 = none; 1 = block-diagonal (block); 2 = learned (net on the grid of
 *        surface, wavenumber k, on top of block if it is not NULL).  With
 *        precond = 2 a block that does not converge or meets a NaN is run again
 *        with precond = 1 from the initial guess (fallback_used).
 * Uses device work memory of about (2 restart + 6) n double2 per right-hand side
 * of a block, allocated stream-ordered and freed before return; synchronises
 * the ctx stream.
 * report[host] (may be NULL): iterations (block iterations, summed over blocks and
 * refinements), final relative residual (max over right-hand sides, from an
 * FP64-accurate product), refinements, fallback, wall time, matrix products.
 * Errors: BIE_EINVAL, BIE_ENOMEM, BIE_ENOCONV, BIE_ENAN (NaN or Inf in the data
 * or the iterates), BIE_ETIMEOUT, BIE_ECUDA.
 * bie_solve: the same for a bare FP64 matrix A [dev] double2[n][n]; it makes the
 * copy prec needs for the duration of the call.                                 */
typedef struct {
  double tol;
  int restart;
  int maxit;
  int prec;
  int precond;
  bie_blockdiag block;   /* precond 1, optional base for 2 */
  bie_net net;           /* precond 2 */
  bie_surface surface;   /* precond 2: the grid and Jacobians of the unknowns */
  double k;              /* precond 2: wavenumber feature */
} bie_solve_opts;
typedef struct {
  int iterations;        /* block iterations (one block product each)          */
  int refinements;       /* outer FP64-accurate refinement steps (prec 1, 2)    */
  double rel_residual;   /* max over right-hand sides                           */
  double seconds;        /* wall time of the call                               */
  int fallback_used;     /* precond = 2 fell back to the block preconditioner   */
  int matvecs;           /* block products with the matrix (all precisions)     */
} bie_solve_report;
bie_status bie_solve_matrix(bie_ctx ctx, bie_matrix M, const double* rhs, int nrhs, double* x,
                            const bie_solve_opts* opts, bie_solve_report* report);
bie_status bie_solve(bie_ctx ctx, int64_t n, const double* A, const double* rhs, int nrhs,
                     double* x, const bie_solve_opts* opts, bie_solve_report* report);

/* ---- boundary data and fields (Section 3.4, Section 5) ---------------------
 * bie_rhs: g on the collocation nodes.  kind 0: plane wave, sound-soft,
 * g = -e^{ik d.x} (param = d[3]); kind 1: point source g = G(x; x_src)
 * (param = x_src[3]), G = e^{ik|x-y|}/(4 pi |x-y|); kind 2: its normal
 * derivative dG/dnu(x) (Neumann data, param = x_src[3]).  g [dev] double2[N]. */
bie_status bie_rhs(bie_ctx ctx, bie_surface s, int kind, const double* param, double k, double* g);

/* bie_field_eval: u(x_p) (far_field = 0) or the far-field pattern u_inf(d_p)
 * (far_field = 1) of the representation rep (BIE_OP_S: single layer;
 * BIE_OP_K: double layer; BIE_OP_CFIE: double layer - i eta single layer)
 * with weighted density [dev] double2[N]; 16-point Gauss-Legendre in t times
 * the trapezoid rule in theta; points assumed well separated from the surface.
 *   pts [dev] double[n][3];  out [dev] double2[n].                            */
bie_status bie_field_eval(bie_ctx ctx, bie_surface s, int rep, double k, double eta,
                          const double* density, const double* pts, int64_t n, int far_field,
                          double* out);

#ifdef __cplusplus
}
#endif
#endif /* BIE_H */
