/*
 * ddi.h -- C ABI of the GB300 NUFFT dipole-dipole interaction (DDI) library.
 *
 * The library evaluates the dipolar potential Phi = U_dip * rho of a density rho given
 * on a uniform grid (Sec. 1, Eqs. DipGPE0 / dipole-poten0 / DipKer; two axes: Eq. dipmn)
 * by the NUFFT method of Sec. 2.1 (Eq. DDI-Trun1): a type-2 NUFFT takes rho to a
 * spherical (3D) or polar (2D) Fourier quadrature, the values are multiplied by the
 * symbol and the quadrature weights, and a type-1 NUFFT sums them back onto the grid.
 * On top of it sit the time-splitting step (Sec. 4.1, Eq. tssp2, Case I), the
 * energies of Sec. 3.2, the normalised gradient flow (Sec. 3.1, Eqs. gf-eq2..gffg33)
 * and the adjoint of the time-splitting step.
 *
 * Conventions shared by every entry point
 *  - Grids are C-ordered [z][y][x] (3D) or [y][x] (2D), x fastest; grid point
 *    j = (jx, jy, jz) sits at x_j = lo + j * h with h_d = len_d / n_d (the periodic
 *    duplicate endpoint of Sec. 4.1 is dropped).
 *  - A plan has a precision: DDI_FP64 (real arrays double, complex arrays interleaved
 *    double pairs) or DDI_FP32 (FP32 arrays and interleaved float pairs; quadrature
 *    nodes, weights and deconvolution factors are built in FP64 and rounded once).
 *  - "Device pointer" arguments must be device memory of the plan's device, laid out
 *    as above, owned by the caller.  "Host pointer" arguments are host memory owned by
 *    the caller (pinned memory is fastest).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Entry points that
 *    only launch work return before it finishes; those that return scalars synchronise
 *    the stream.
 *  - Every entry point returns a ddi_status; no exception or abort crosses the ABI.
 *    Arguments are validated before any launch; ddi_last_error() then describes the
 *    failure (thread-local string, valid until the next call on that thread).
 */
#ifndef DDI_GB300_H
#define DDI_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DDI_OK = 0,
  DDI_ERR_ARG = -1,        /* invalid argument (sizes, axes, pointers, precision) */
  DDI_ERR_CUDA = -2,       /* a CUDA runtime call or kernel launch failed */
  DDI_ERR_OOM = -3,        /* a device or host allocation failed (plan or batch creation) */
  DDI_ERR_NONFINITE = -4,  /* NaN/Inf found in an input or produced by an iteration */
  DDI_ERR_TIMEOUT = -5,    /* a bounded device-side wait gave up */
  DDI_ERR_NOCONV = -6,     /* an iteration hit its step limit before the tolerance */
  DDI_ERR_INTERNAL = -7    /* an unexpected host-side failure inside the library */
} ddi_status;

enum { DDI_FP64 = 0, DDI_FP32 = 1 };

typedef struct ddi_plan_s* ddi_plan;
typedef struct ddi_batch_s* ddi_batch;

/* ddi_batch_create flags */
enum { DDI_BATCH_GRAPH = 1, DDI_BATCH_AUTOTUNE = 2 };

/* Plan descriptor.  Zero fields take the defaults listed. */
typedef struct {
  int dim;             /* 2 or 3 */
  int n[3];            /* grid sizes (x, y, z); powers of two, 8..1024 (3D: <= 512); n[2] = 1 in 2D */
  double lo[3];        /* lower box corner per axis */
  double len[3];       /* box length per axis (> 0) */
  double axis_n[3];    /* dipole axis n (unit vector; Eq. DipKer).  In 2D n_perp = (n0, n1), n3 = n2 */
  double axis_m[3];    /* second axis m (Eq. dipmn); all zero => m = n */
  int nr, ntheta, nphi;/* quadrature sizes; 0 => (N, N/2, N) in 3D, (2N, -, 2N) in 2D, N = max n */
  double kmax;         /* radius R of the Fourier ball; 0 => pi / min_d h_d */
  int precision;       /* DDI_FP64 or DDI_FP32 */
  double nufft_tol;    /* requested NUFFT tolerance; 0 => 1e-13 (FP64) / 1e-6 (FP32) */
  int tile[3];         /* spread tile (x, y, z) in fine cells, >= w - 1 and dividing 2n (rounded to
                          such a size); 0 => built-in choice; tile[0] < 0 => picked by the
                          spread-tile autotuner (ddi_tune_spread_tile) when the plan is created */
  int chunk;           /* max nodes per spread work item; 0 => built-in choice */
  double split_k0;     /* 3D only.  0 => the quadrature of Eq. DDI-Trun1 on the ball |k| <= kmax.
                          != 0 => the improved split algorithm of Sec. 2.1 (Eq. 3.9) with the window
                          q(k) = exp(-|k|^2 / k0^2), k0 = split_k0 (< 0 => k0 = 9.6 / min_d len_d: the
                          smooth part's kernel decays like exp(-(k0 r)^2 / 4), ~1e-10 at the distance
                          len_d that the 2x zero padding puts between a point and the nearest
                          periodic image of the box):
                            Phi = I_1 + I_2,
                            I_1 = Re IFFT[ p(k_l) FFT[rho zero-padded to the 2n fine grid] ], cropped,
                                  p = (1 - q) Uhat, on the fine grid's modes k_l = 2 pi l / (2 len);
                            I_2 = the quadrature sum of Eq. DDI-Trun1 on the small ball
                                  |k| <= kmax (0 => 6 k0) with weights W_q q(k_q), by the NUFFT.
                          Quadrature sizes 0 => nr = 0.48 K, ntheta = 0.32 K, nphi = 0.64 K, each
                          rounded up to a multiple of 8 and at least (16, 8, 16), K = kmax times the
                          box diagonal (the phase range of e^{ik.x} the ball rule has to resolve). */
  int ellipsoid;       /* 0 => the rule on the ball |k| <= kmax.  1 => the same rule mapped onto the
                          ellipsoid with semi-axes kmax e_d, e_d = min h / h_d (pi / h_d by default), for
                          heterogeneous boxes such as the thin domains D_eps of Sec. 2.1 (h_z = eps h_x):
                          nodes e * (r khat), Jacobian e_x e_y (e_z), symbol at the direction of k, and
                          in 2D the symbol's factor |k| = r |e * khat|.  Default polar (3D) / azimuthal
                          (2D) size ceil(N/2 ratio) / 2 ceil(N ratio), ratio = max h / min h.  Not
                          combined with split_k0. */
  int split_full_passes; /* split plans: 0 => the ball's type-2 / type-1 NUFFT runs its y and z fine-grid
                          passes only on the lines through its taps (|l_d| <= kmax h_d nf_d / (2 pi) +
                          w/2 + 2 around k = 0; the other lines are zero or never read); 1 => on
                          every line, as a plan without split_k0 does */
  int spread;          /* type-1 spreading scheme: 0 => automatic (columns where they apply, else plane
                          tiles); DDI_SPREAD_TILES => owner-computes tile planes in shared memory (`tile`,
                          `chunk`); DDI_SPREAD_COLUMNS => columns of the fine grid whose planes along the
                          last axis a warp accumulates in registers: 8 x 8 cells in x-y running along z
                          (3D), 8 cells in x running along y (2D).  Applies to FP32 plans whose fine grid
                          is a multiple of 8 in x (3D: and in y) and at least w + 7 cells in x (3D: w + 7
                          in y and w in z; 2D: w in y), and not to compensated 2D plans; DDI_ERR_ARG
                          otherwise; `chunk` = visits per work item */
  int check_finite;    /* NaN / Inf in rho: the pad pass of every evaluation records them in a device
                          flag of the plan (at no cost for finite input).  0 => ddi_apply stays
                          asynchronous and the flag is read by ddi_plan_check (and by ddi_apply_host,
                          which synchronises anyway); 1 => ddi_apply also synchronises `stream` and
                          returns DDI_ERR_NONFINITE when its input held a non-finite value */
  int compensated;     /* FP32 plans: 1 => compensated arithmetic in the quadrature sum's NUFFT: the column
                          spread accumulates each fine cell with Kahan summation and the fine-grid FFT passes
                          apply the twiddles as FP32 head + tail; 0 => plain FP32 (the default: on the
                          128^3 workload both give the same error to 1e-7, which the w = 8 kernel's
                          truncation and the FFTs' roundoff set, and the compensated spread is slower) */
} ddi_plan_desc;

enum { DDI_SPREAD_AUTO = 0, DDI_SPREAD_TILES = 1, DDI_SPREAD_COLUMNS = 2 };

/* Read-only facts about a built plan (sizes and the NUFFT parameters chosen). */
typedef struct {
  int dim, precision;
  int n[3];
  int nf[3];           /* oversampled (fine) grid, 2 n per axis */
  int width;           /* exponential-of-semicircle kernel width in fine cells */
  double beta;         /* kernel shape parameter */
  int64_t nodes;       /* quadrature nodes M (the full, antipodally closed set) */
  int64_t nodes_used;  /* nodes processed per NUFFT (M/2: one of each +-k pair) */
  int tile[3];
  int spread_items, spread_split_tiles, interp_items;
  double kmax;
  int nr, ntheta, nphi;
  size_t device_bytes; /* device memory held by the plan */
  double spread_tuned_ms; /* spread time of the tile the autotuner picked, in ms; 0 if not tuned */
  double split_k0;     /* window width k0 of the split algorithm; 0 if the plan does not split */
  int ellipsoid;       /* 1 if the quadrature is the ellipsoidal rule */
  int band[2];         /* split plans: half-widths (x, y) of the band of fine-grid lines the ball's
                          y and z passes transform (0, 0: every line) */
  int spread;          /* DDI_SPREAD_TILES or DDI_SPREAD_COLUMNS: the scheme the plan uses (0 from
                          ddi_plan_describe) */
  int yrange[2];       /* first fine-grid y line and number of lines (cyclic) that hold node taps; the
                          NUFFT's z passes transform only their columns (0, 0 from ddi_plan_describe) */
} ddi_plan_info;

/* Energies of Sec. 3.2 for a state phi (all FP64). */
typedef struct {
  double E, mu, Ekin, Epot, Eint, Edip, virial, mass;
  int steps;           /* gpe_ground_state: outer steps taken */
  int inner_max;       /* gpe_ground_state: largest inner iteration count of any step */
  double last_change;  /* gpe_ground_state: |E^{n+1} - E^n| or max|phi^{n+1}-phi^n|/dt at exit */
} gpe_stats;

enum { GPE_STOP_ENERGY = 0, GPE_STOP_PAPER = 1 };

/* ---- status ---------------------------------------------------------------- */
const char* ddi_status_str(int status);   /* static string for a status code */
const char* ddi_last_error(void);         /* detail of the last failure on this thread */

/* ---- quadrature tables (host only, no GPU needed) --------------------------- */
/* Sec. 2.1, Eq. DDI-Trun1: nodes k_q and weights W_q of the discrete sum
 *   Phi_j = Re sum_q W_q e^{i k_q.x_j} h^d sum_j' rho_j' e^{-i k_q.x_j'}.
 * Rule: n_r-point Gauss-Legendre radial on [0, R], n_theta-point Gauss-Legendre in
 * cos(theta), n_phi-point trapezoid azimuth whose second half is the exact negation
 * of the first; W_q = w_q |k|^{d-1} Uhat(k_q) / (2 pi)^d.  Node order
 * q = (i_r n_theta + j_u) n_phi + m (3D), i_r n_phi + m (2D).
 * k: [M][dim] doubles, W: [M] doubles, l0: [M][dim] int32 (first fine-grid tap,
 * ceil(k_d h_d nf_d / (2 pi) - w/2), before wrapping), each may be NULL.  Call with
 * all three NULL to get *M only.  Host pointers. */
int ddi_quadrature_tables(const ddi_plan_desc* desc, int64_t* M, double* k, double* W,
                          int32_t* l0);

/* ---- plans ------------------------------------------------------------------ */
/* Build a plan on the current device: quadrature, NUFFT tables, node binning, spread
 * work list and all device workspace (fine grid, node arrays, GPE buffers).  The
 * only call that allocates.  `stream` orders the table uploads. */
int ddi_plan_create(ddi_plan* out, const ddi_plan_desc* desc, void* stream);
int ddi_plan_destroy(ddi_plan plan);
int ddi_plan_get_info(ddi_plan plan, ddi_plan_info* info);
/* What ddi_plan_create would build from `desc`, without building it (host only, no GPU
 * needed): the normalised sizes, fine grid, kernel width and shape, node counts, kmax,
 * quadrature sizes, split_k0, ellipsoid and band.  Fields that depend on the device build
 * (tile, spread work items, device_bytes, spread_tuned_ms) are 0.  DDI_ERR_ARG for an invalid
 * descriptor (as ddi_plan_create) or a NULL info. */
int ddi_plan_describe(const ddi_plan_desc* desc, ddi_plan_info* info);

/* ---- the DDI (Sec. 2.1) -------------------------------------------------------- */
/* Phi = U_dip * rho by the quadrature sum above, through the NUFFT: deconvolve and
 * pad rho into the 2x oversampled grid, FFT, interpolate at one node of each +-k pair,
 * multiply by 2 h^d W_q, spread, inverse FFT, crop, deconvolve, real part.
 * rho, phi: device pointers to n-sized real grids in the plan precision; may alias.
 * Non-finite values in rho are recorded (see ddi_plan_desc.check_finite, ddi_plan_check);
 * with check_finite = 1 the call synchronises and returns DDI_ERR_NONFINITE for them. */
int ddi_apply(ddi_plan plan, const void* rho, void* phi, void* stream);

/* Same, end to end from host memory: copies rho in, applies, copies phi out, and
 * synchronises `stream`.  rho_host / phi_host: host pointers (pinned recommended).
 * DDI_ERR_NONFINITE when rho held NaN or Inf (phi is then not meaningful). */
int ddi_apply_host(ddi_plan plan, const void* rho_host, void* phi_host, void* stream);

/* Synchronises `stream`, then reports whether any evaluation of the plan since the last
 * check (or since creation) read a NaN or Inf in its rho: DDI_ERR_NONFINITE (and clears the
 * record) or DDI_OK.  The input check of Sec. 3's iterations applied to the DDI's input. */
int ddi_plan_check(ddi_plan plan, void* stream);

/* ddi_apply with a CUDA event recorded on `stream` after every kernel launch; on
 * return (the stream is synchronised) names[i] / ms[i] hold the i-th launch's kernel
 * name (static string) and its duration in milliseconds, *count the number of launches
 * (at most `cap`).  Same arguments and result as ddi_apply; used by benchmarks to time
 * single kernels on the stream they run on. */
int ddi_apply_timed(ddi_plan plan, const void* rho, void* phi, void* stream, const char** names, double* ms,
                    int cap, int* count);

/* Type-2 stage alone (for tests): f_q for the nodes in the plan's processing order,
 * scaled as the path uses them, c_q = 2 h^d W_q f_q.  c: device pointer to
 * nodes_used complex values; order: ddi_plan_node_order(). */
int ddi_type2(ddi_plan plan, const void* rho, void* c, void* stream);
/* Type-1 stage alone: phi_j = Re sum_q c_q e^{i k_q.x_j} (plan order, nodes_used). */
int ddi_type1(ddi_plan plan, const void* c, void* phi, void* stream);
/* Original node index q (0..M-1) of each processed node, host pointer [nodes_used]. */
int ddi_plan_node_order(ddi_plan plan, int64_t* q);

/* New dipole axes for an existing plan (time-dependent axes n(t), m(t), Eq. dipole-time,
 * Sec. 3; two axes, Eq. dipmn): rebuilds the node scales 2 h^d W_q for the symbol of
 * (axis_n, axis_m) in one FP64 pass on the device, with the operations of the plan
 * builder in the same order, so the plan then computes exactly what a plan created with
 * these axes computes (bit for bit).  axis_n: host pointer to 3 doubles (unit vector;
 * 2D: n_perp = (n0, n1), n3 = n2); axis_m: 3 doubles or NULL for m = n.  Asynchronous on
 * `stream` (later calls on the plan see the new axes); DDI_ERR_ARG for a non-unit axis. */
int ddi_plan_set_axes(ddi_plan plan, const double* axis_n, const double* axis_m, void* stream);

/* ---- GPE (Secs. 3-4) -------------------------------------------------------------- */
/* nsteps Strang steps of Eq. tssp2, Case I (f = 0, sigma = 1, fixed axis):
 * psi <- K N K psi with K = F^{-1} exp(-i dt |mu|^2/4) F and
 * N: psi <- psi exp(-i dt (V + beta |psi|^2 + lambda Phi(|psi|^2))), Phi by ddi_apply.
 * psi: device complex grid (in place); V: device real grid. */
int gpe_step(ddi_plan plan, void* psi, const void* V, double beta, double lambda,
             double dt, int nsteps, void* stream);

/* Nonlinearity and damping of Eq. DipGPE1 (Sec. 5): beta |psi|^(2 sigma) and
 * -i f(|psi|^2) psi with f = 0 (GPE_DAMP_NONE, Case I), f = delta (GPE_DAMP_LINEAR, Case II,
 * inelastic collisions with the background gas) or f = delta rho^q (GPE_DAMP_POWER, Case III;
 * q = 1 two-body, q = 2 three-body loss). */
enum { GPE_DAMP_NONE = 0, GPE_DAMP_LINEAR = 1, GPE_DAMP_POWER = 2 };
typedef struct {
  double sigma;  /* > 0: 1 cubic, 2 quintic */
  int damping;   /* GPE_DAMP_* */
  double delta;  /* > 0 when damped */
  double q;      /* > 0, GPE_DAMP_POWER only */
} gpe_nonlinearity;

/* nsteps Strang steps of Eq. tssp2 for Eq. DipGPE1 with a fixed dipole axis: the nonlinear
 * sub-step psi2 = psi1 exp(-i [dt V + H + lambda U_dip * g]) exp(-F) is integrated exactly,
 * with H = beta int_0^dt h^sigma, F = int_0^dt f(h), g = int_0^dt h (Eqs. fun1, fun2;
 * h(phi, tau) the density under the damping alone) in the closed forms of Cases I-III.
 * Arguments as gpe_step; nl: host pointer.  The mass decays by Eq. Mass_Disp when damped.
 * DDI_ERR_ARG for out-of-range parameters. */
int gpe_step_ex(ddi_plan plan, void* psi, const void* V, double beta, double lambda,
                const gpe_nonlinearity* nl, double dt, int nsteps, void* stream);

/* Energies of Sec. 3.2 (E_kin spectral, FP64 reductions), mu = E + E_int + E_dip,
 * virial I = 2E_kin - 2E_pot + 3E_int + 3E_dip (Eq. vir_iden), mass.  Synchronises. */
int gpe_energy(ddi_plan plan, const void* psi, const void* V, double beta, double lambda,
               gpe_stats* out, void* stream);

/* Normalised gradient flow, backward Euler (Eqs. gf-eq2..gffg33); the implicit
 * equation is solved by the stabilised fixed point
 *   phi1 <- F^{-1}[F(phi/dt + (alpha - W) phi1) / (1/dt + alpha + |mu|^2/2)],
 * W = V + beta|phi|^2 + lambda Phi, alpha = (max W + min W)/2, until
 * max|change| <= inner_tol (or 200 sweeps), then phi <- phi1/||phi1||.
 * Stops when rule = GPE_STOP_ENERGY: |E^{n+1} - E^n| < tol, GPE_STOP_PAPER:
 * max|phi^{n+1}-phi^n|/dt <= tol (Sec. 3.2); checked every `check_every` steps.
 * Returns DDI_ERR_NOCONV when max_steps is reached.  phi: device complex grid, in
 * place (normalised on entry).  Synchronises. */
int gpe_ground_state(ddi_plan plan, void* phi, const void* V, double beta, double lambda,
                     double dt, double tol, int rule, double inner_tol, int max_steps,
                     int check_every, gpe_stats* out, void* stream);

/* Adjoint of one gpe_step step (nsteps = 1) for the pairing Re h^d sum conj(a) b.
 * psi_in: the step's input state (device, read only; the step is recomputed);
 * cot: device complex grid holding dJ/dpsi_out on entry, dJ/dpsi_in on exit;
 * grad_V: device real grid, incremented by h^d r with r = Re(conj(-i dt psi2) g2)
 * (the step's contribution to dJ/dV_j).  One DDI of r (Phi is self-adjoint). */
int gpe_step_adjoint(ddi_plan plan, const void* psi_in, void* cot, void* grad_V,
                     const void* V, double beta, double lambda, double dt, void* stream);

/* Gradient of a final-time observable with respect to the trap (the differentiable dynamics
 * of Sec. 4.1, Eq. tssp2): J = h^d sum_j x_j^2 |psi_T,j|^2, x the coordinate along the grid's
 * last axis (z in 3D, y in 2D; x_j = lo + j h), psi_T after nsteps gpe_step steps (each a
 * full Strang step) from psi0 with trap V.
 * gpe_trap_observable: the forward run alone.  psi0: device complex grid (read only);
 *   psi_T: device complex grid receiving the final state (distinct from psi0); J: host
 *   pointer.  Synchronises.
 * gpe_trap_gradient: J and dJ/dV (grad_V: device real grid, overwritten) by the adjoint of
 *   every step (gpe_step_adjoint), with checkpointed recomputation: the forward sweep keeps
 *   the state every `checkpoint` steps, the backward sweep recomputes each segment's step
 *   inputs from its checkpoint; the seed cotangent 2 x^2 psi_T and J are formed on the
 *   device.  work: device buffer of the caller, at least gpe_trap_gradient_workspace bytes
 *   (ceil(nsteps / checkpoint) + checkpoint + 2 complex grids).  Synchronises.
 * DDI_ERR_ARG for NULL pointers, nsteps or checkpoint < 1, a short workspace;
 * DDI_ERR_NONFINITE when J is not finite. */
int gpe_trap_observable(ddi_plan plan, const void* psi0, const void* V, double beta, double lambda, double dt,
                        int nsteps, void* psi_T, double* J, void* stream);
int gpe_trap_gradient_workspace(ddi_plan plan, int nsteps, int checkpoint, size_t* bytes);
int gpe_trap_gradient(ddi_plan plan, const void* psi0, const void* V, double beta, double lambda, double dt,
                      int nsteps, int checkpoint, void* work, size_t work_bytes, double* J, void* grad_V,
                      void* stream);

/* ---- batches ---------------------------------------------------------------------- */
/* Many DDI evaluations (Sec. 2.1, Eq. DDI-Trun1) in one call: item i has its own grid,
 * box, dipole axes, quadrature and precision (descs[i], as for ddi_plan_create) and
 * computes phi[i] = U_dip,i * rho[i] exactly as ddi_apply does with a plan built from
 * descs[i] (bit-identical for the same spread tile).  The items run concurrently on the
 * batch's own side streams, forked from and joined back into `stream`.
 * Flags: DDI_BATCH_GRAPH records the launches of all items into one CUDA graph on the
 *   first ddi_batch_apply and replays it (one cudaGraphLaunch) while the rho/phi
 *   pointers stay the same; new pointers re-record it.
 *   DDI_BATCH_AUTOTUNE picks every item's spread tile with the autotuner (also done for
 *   items whose desc.tile[0] < 0): the spread is timed on the item's node set for a few
 *   candidate tiles on this device and the fastest kept; results are cached per grid and
 *   quadrature shape for the life of the process, so each shape is timed once.
 * ddi_batch_create builds all plans (host threads; allocates all device memory, none for
 * the GPE) and synchronises `stream`.  count >= 1.  Errors: DDI_ERR_ARG for an invalid
 * descriptor (ddi_last_error names the item), DDI_ERR_OOM, DDI_ERR_CUDA. */
int ddi_batch_create(ddi_batch* out, const ddi_plan_desc* descs, int count, int flags, void* stream);
/* Synchronises the device, then frees the batch (NULL is a no-op). */
int ddi_batch_destroy(ddi_batch batch);
/* Number of items (0 for NULL). */
int ddi_batch_size(ddi_batch batch);
/* Facts about item `item`'s plan (tile chosen, nodes, device bytes). */
int ddi_batch_get_info(ddi_batch batch, int item, ddi_plan_info* info);
/* rho, phi: host arrays of ddi_batch_size() device pointers, item i's grids in its
 * precision; rho[i] may alias phi[i], distinct items must not share memory.
 * Asynchronous on `stream`.  Calls on one batch must not overlap on the GPU (the items'
 * workspaces are reused). */
int ddi_batch_apply(ddi_batch batch, const void* const* rho, void* const* phi, void* stream);
/* How often the graph was recorded and launched (DDI_BATCH_GRAPH); either may be NULL. */
int ddi_batch_graph_stats(ddi_batch batch, long long* records, long long* launches);

/* ---- without allocation -------------------------------------------------------------- */
/* The paper has no counterpart to this call: it serves callers that cannot allocate
 * device memory (a host whose pool reserves the whole device, a plugin that may only use
 * memory it is handed, a loop that must not risk the synchronisation an allocation can
 * cause).  It computes the FP64 sums behind gpe_energy,
 *   sums[0] = sum |psi|^2, sums[1] = sum V |psi|^2, sums[2] = sum |psi|^4
 * (multiply by h^d, beta h^d / 2 for the energies), over `count` grid points.  psi:
 * device complex array (interleaved, FP64 or FP32 per `precision`), V: device real
 * array, sums: device pointer to 3 doubles, all owned by the caller.  Allocates nothing:
 * its block partials live in a fixed 512 KiB device array of the library, shared by all
 * calls, so count is limited to 2^26 (DDI_ERR_ARG beyond).  The first call on each
 * device looks the array up (cudaGetSymbolAddress) and should come before any stream
 * capture.  Calls that overlap on the GPU race on the shared array.  Asynchronous on
 * `stream`. */
int gpe_sums_noalloc(const void* psi, const void* V, int64_t count, int precision, double* sums,
                     void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DDI_GB300_H */
