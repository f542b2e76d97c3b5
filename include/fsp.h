/*
 * fsp.h -- C ABI of libfsp, the GB300 (sm_103a) implementation of the WENO
 * interpolation-based, upwind-biased, free-stream-preserving (WENOIU) schemes of
 * Q. Li and D. Sun, arXiv:1810.11103, for the 2-D compressible Euler equations on
 * structured curvilinear grids.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid.  Nodes (i, j), 0 <= i < ni, 0 <= j < nj, i fastest; unit computational
 *   spacing.  Coordinates x, y: device arrays of nj * ni doubles, node (i, j) at
 *   [j * ni + i].
 * State.  Conservative Q = (rho, rho u, rho v, E), E = p/(gamma-1) + rho |u|^2 / 2
 *   (Eq. 2.1 in two dimensions): 4 planes, plane v at Q + v * nj * ld, node (i, j) at
 *   [j * ld + i]; ld >= ni.  Element type double (FSP_FP64) or float (FSP_FP32,
 *   FSP_FP32_MIXED).
 *   The same layout holds for dQ/dt, Q_bar and every other state-shaped array.
 * Metrics.  5 planes of doubles (xi_x^, xi_y^, eta_x^, eta_y^, J^-1) on the grid
 *   extended by FSP_G ghost layers on each side: plane p, node (i, j) with
 *   -FSP_G <= i < ni + FSP_G, -FSP_G <= j < nj + FSP_G, at
 *   [p * (nj + 2 FSP_G) * (ni + 2 FSP_G) + (j + FSP_G) * (ni + 2 FSP_G) + (i + FSP_G)].
 *   fsp_metrics_elems() gives the count.
 * Boundaries.  Faces 0..3 = i-min, i-max, j-min, j-max.  Ghost states are formed
 *   inside the kernels (no ghost storage for Q): periodic wraps; transmissive copies
 *   the boundary node; Dirichlet uses bc_state[face]; slip wall mirrors about the
 *   boundary node and reverses the velocity along the boundary node's grid normal;
 *   far field takes bc_state[face] where its velocity enters through the face and is
 *   transmissive elsewhere.  Ghost coordinates: periodic wrap plus the period vector,
 *   otherwise odd reflection x_{-k} = 2 x_0 - x_k.  Periodic faces come in pairs; a
 *   non-periodic direction needs at least 9 nodes.
 * Memory.  All array arguments are device pointers owned by the caller.  The library
 *   allocates nothing; calls needing scratch take a caller-provided workspace `ws` of
 *   at least fsp_workspace_size() bytes (256-byte aligned).
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Every call only enqueues work on it and returns; results are ready after the
 *   caller synchronises the stream.
 * Errors.  Every entry point returns an fsp_status and never aborts.  Arguments are
 *   checked on the host before anything is enqueued (FSP_ERR_INVALID_ARG; host or
 *   unregistered pointers are rejected); launch failures return FSP_ERR_CUDA.
 *   Asynchronous device faults surface at the caller's next synchronisation.
 * Threads.  No global mutable state except where stated; distinct calls may run on
 *   distinct streams concurrently if their output and workspace buffers differ.
 */
#ifndef FSP_H
#define FSP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FSP_G 4 /* ghost layers of the stored metrics */

typedef enum {
  FSP_OK = 0,
  FSP_ERR_INVALID_ARG = 1,
  FSP_ERR_UNSUPPORTED = 2,
  FSP_ERR_CUDA = 3,
  FSP_ERR_NONFINITE = 4,
  FSP_ERR_TIMEOUT = 5,
  FSP_ERR_NOMEM = 6
} fsp_status;

/* Schemes of Section 3: third- and fifth-order, one or two midpoints; and the seventh-order
 * one-midpoint scheme of the Appendix (scheme (1) with alpha = 1: Table A1 candidates, the
 * fourth-order mapping, an eighth-order central operator and eight-point midpoint metrics;
 * its smoothness indicators are those of Eq. 3.22's definition applied to the cubics of
 * Table A1).  The adjoint entry points cover these five. */
/* FSP_WENOIU7_4MP: the Appendix's scheme (3), four midpoints j - 3/2 .. j + 3/2 in h+ and an
 * eighth-order central operator with midpoint terms to 5/2.  Its midpoint fluxes reach from
 * j - 5/2 to j + 5/2, six nodes beyond a face, while every stored array carries FSP_G = 4 ghost
 * layers: it is built for periodic blocks (ghost metrics wrap) in FP64 and FP32 through the
 * single-block entry points; other faces, FSP_FP32_MIXED, the batch, the adjoint and the
 * three-dimensional path return FSP_ERR_UNSUPPORTED. */
enum { FSP_WENOIU3_1MP = 0, FSP_WENOIU3_2MP = 1, FSP_WENOIU5_1MP = 2, FSP_WENOIU5_2MP = 3, FSP_WENOIU7_1MP = 4,
       FSP_WENOIU7_4MP = 5 };
/* Arithmetic of the right-hand side.  Metrics are FP64 in every mode.
 * FSP_FP64        everything in double.
 * FSP_FP32        state, WENO and fluxes in float (metrics rounded to float on load); the
 *                 free-stream residual is at FP32 round-off.
 * FSP_FP32_MIXED  state, characteristic projection and WENO in float; metric products,
 *                 fluxes, the h combination and the difference in double, so the
 *                 free-stream residual stays at FP64 round-off.  State arrays are float. */
enum { FSP_FP64 = 0, FSP_FP32 = 1, FSP_FP32_MIXED = 2 };
enum { FSP_BC_PERIODIC = 0, FSP_BC_TRANSMISSIVE = 1, FSP_BC_DIRICHLET = 2, FSP_BC_SLIPWALL = 3,
       FSP_BC_FARFIELD = 4, FSP_BC_LINK = 5 /* multi-block only: see fsp_batch_create */ };

typedef struct {
  int scheme;          /* FSP_WENOIU*                                                   */
  int precision;       /* FSP_FP64 or FSP_FP32                                          */
  int interp;          /* midpoint interpolation of nodal metrics and coordinates:
                          0 = central Lagrange, 4 points (third order) or 6 points
                          (fifth order); 1 = two-point average (Section 2.4)           */
  int ppm;             /* 1 = piecewise-polynomial mapping of the weights (Eqs. 3.15,
                          3.23); 0 = plain weights (Eqs. 3.12-3.13)                    */
  int linear_weights;  /* 1 = omega_k = C_k (linear interpolation, no mapping)          */
  int bc[4];           /* FSP_BC_* per face                                            */
  double gamma;        /* ratio of specific heats (1.4)                                */
  double lf_alpha;     /* alpha of the Lax-Friedrichs-type splitting, 1.1-1.2 (Sec. 2.3) */
  double eps;          /* epsilon of Eq. (3.13): 1e-40 with the mapping, else 1e-6     */
  double bc_state[4][4]; /* conservative state per face (Dirichlet, far field)         */
  /* Options beyond the schemes the paper tests (Section 7 names them; the free parameter is
   * the alpha of Eqs. 3.5 and 3.17 and of the Appendix's scheme (1)).  All zero = the paper's
   * schemes.  The adjoint entry points and the batch's marching tile variants take only the
   * defaults.                                                                             */
  int weights;         /* 0 = the weights of Eqs. 3.12-3.13 (with ppm); 1 = WENO-Z weights
                          C_k (1 + (tau/(eps + IS_k))^2), tau = |IS_0 - IS_{r-1}| (r = 2, 3)
                          or |IS_0 + 3 IS_1 - 3 IS_2 - IS_3| (r = 4), no mapping          */
  int mid_split;       /* splitting of the midpoint flux f_{j+1/2}: 0 = Lax-Friedrichs type
                          (Section 2.3), 1 = Steger-Warming, 2 = Van Leer; FSP_FP64 and
                          FSP_FP32 only                                                    */
  double scheme_alpha; /* free parameter of the one-midpoint schemes (WENOIU3-1MP, -5-1MP,
                          -7-1MP); 0 or 1 = the printed schemes; any other value > 0 for a
                          one-midpoint scheme only; the metrics use the scheme's own central
                          operator                                                        */
} fsp_config;

typedef struct {
  int ni, nj;          /* nodes per direction                                          */
  long long ld;        /* row stride of Q-shaped arrays, elements (>= ni)              */
  double period[2][2]; /* (dx, dy) added to the coordinates per wrap in i, then in j    */
} fsp_block;

/* Human-readable text of a status code (static storage). */
const char* fsp_status_string(fsp_status s);

/* Number of doubles of a metrics array for this block: 5 (nj + 8)(ni + 8). */
size_t fsp_metrics_elems(const fsp_block* blk);

/* Bytes of workspace needed by fsp_rhs, fsp_rk3_step, fsp_cfl_dt and the VJPs. */
fsp_status fsp_workspace_size(const fsp_config* cfg, const fsp_block* blk, size_t* bytes);

/*
 * fsp_metrics -- conservative grid metrics (Eq. 2.3 in 2-D: xi_x^ = y_eta,
 * xi_y^ = -x_eta, eta_x^ = -y_xi, eta_y^ = x_xi) and Jacobian (Eq. 2.5, whose 2-D form is
 * J^-1 = x_xi y_eta - x_eta y_xi).  Every derivative uses the scheme's central operator
 * delta^{c,(1)} (Eq. 2.7; Eqs. 3.7, 3.9, 3.19, 3.21) along its direction, with midpoint
 * values from the interpolation chosen by cfg->interp (Section 2.4).  Computed on the
 * node range extended by FSP_G ghost layers.  x, y: nj*ni doubles; metrics: output,
 * fsp_metrics_elems() doubles.  FP64 regardless of cfg->precision.
 */
fsp_status fsp_metrics(const fsp_config* cfg, const fsp_block* blk, const double* x,
                       const double* y, double* metrics, void* stream);

/*
 * fsp_line_lambda -- the per-line maxima behind A^ of the Lax-Friedrichs-type splitting
 * (Section 2.3): for each grid line the maximum over its interior nodes of
 * |U^| + c |k^|, with U^ = k_x^ u + k_y^ v and k^ the line's own metric pair; the
 * splitting uses A^ = lf_alpha * maximum.  lam_xi: nj doubles (one per row, direction
 * xi); lam_eta: ni doubles (one per column).  Output buffers are overwritten.
 */
fsp_status fsp_line_lambda(const fsp_config* cfg, const fsp_block* blk, const double* metrics,
                           const void* Q, double* lam_xi, double* lam_eta, void* stream);

/*
 * fsp_rhs -- the semi-discrete right-hand side dQ/dt = -(dE^/dxi + dF^/deta) / J^-1 of
 * Eq. (2.2) on a stationary grid.  Per direction: the split fluxes f+- = (E^ +- A^ Q)/2
 * at the nodes (Section 2.3); at every midpoint the state interpolated from each side by
 * characteristic WENO (Eqs. 3.10-3.13 with Table 1, indicators of Eq. 3.22, mapping
 * 3.15/3.23, projection of Section 3.4), split with the interpolated midpoint metrics;
 * the upwind-biased combination h = h+ + h- of Eq. (3.4), (3.8), (3.16) or (3.20); and
 * the difference of Eq. (3.2).  Q: input state; dQdt: output (same layout, may not alias
 * Q); ws: workspace.
 */
fsp_status fsp_rhs(const fsp_config* cfg, const fsp_block* blk, const double* metrics,
                   const void* Q, void* dQdt, void* ws, size_t ws_bytes, void* stream);

/*
 * fsp_rhs_noalloc -- the same right-hand side as fsp_rhs, for callers that cannot
 * allocate device memory (no workspace argument).  The paper has no counterpart: this is
 * a convenience of the library.  It suits a solver plugin inside an application that owns
 * every device allocation, a real-time loop where cudaMalloc/cudaFree would synchronise
 * the device, or a caller without an allocator of its own.  Its scratch (per-line maxima
 * and the xi accumulator) lives in one fixed device array of FSP_NOALLOC_SCRATCH_BYTES
 * inside the library, which every GPU that loads the library holds until the process
 * exits.  Limits and behaviour:
 *   - FP64 only (FSP_ERR_UNSUPPORTED otherwise);
 *   - the block must fit: 8 (ni + nj) bytes, rounded up to 256, plus 32 nj ld bytes
 *     <= FSP_NOALLOC_SCRATCH_BYTES, else FSP_ERR_NOMEM and nothing is enqueued;
 *   - the first call on a device looks up the array's device address (this may load the
 *     module), so make that first call before any stream capture;
 *   - all calls share the one array: calls that overlap on the GPU (other streams, other
 *     host threads on the same device) race and must be serialised by the caller;
 *   - the array keeps the previous call's contents; each call clears what must start at
 *     zero.
 * It calls no cudaMalloc, cudaFree or allocating library routine.
 */
#define FSP_NOALLOC_SCRATCH_BYTES (8u << 20)
fsp_status fsp_rhs_noalloc(const fsp_config* cfg, const fsp_block* blk, const double* metrics,
                           const void* Q, void* dQdt, void* stream);

/*
 * fsp_flux_difference -- one direction of the right-hand side: at every node the
 * difference H_{s+1/2} - H_{s-1/2} (Eq. 3.2, unit spacing) along direction dir (0 = xi
 * along i, 1 = eta along j), with h = h+ + h- built exactly as in fsp_rhs and
 * A^ = lf_alpha * lam[line].  lam: the per-line maxima of fsp_line_lambda for that
 * direction (nj values for xi, ni for eta).  mode 0: D <- the difference; mode 1:
 * D <- -(acc + difference) / J^-1, which is dQ/dt when acc holds the other direction's
 * difference.  acc (mode 1 only) and D have the state layout; D may not alias Q or acc.
 * Element types: the difference and acc are double (FSP_FP64, FSP_FP32_MIXED) or float
 * (FSP_FP32); dQ/dt (mode 1) has the state's type.
 * fsp_rhs is fsp_line_lambda + this call for xi (mode 0) + this call for eta (mode 1).
 */
fsp_status fsp_flux_difference(const fsp_config* cfg, const fsp_block* blk, const double* metrics,
                               const void* Q, const double* lam, int dir, int mode, const void* acc,
                               void* D, void* stream);

/*
 * fsp_rk3_step -- one step of the third-order TVD Runge-Kutta scheme (Section 6),
 * Shu-Osher form Q1 = Q + dt R(Q); Q2 = 3/4 Q + 1/4 (Q1 + dt R(Q1));
 * Q <- 1/3 Q + 2/3 (Q2 + dt R(Q2)), with R = fsp_rhs.  Q is updated in place.
 */
fsp_status fsp_rk3_step(const fsp_config* cfg, const fsp_block* blk, const double* metrics,
                        void* Q, double dt, void* ws, size_t ws_bytes, void* stream);

/*
 * fsp_cfl_dt -- the time step cfl / max over interior nodes of
 * [(|U^_xi| + c |grad xi^|) + (|U^_eta| + c |grad eta^|)] / J^-1, written to the device
 * double *dt_out.  (The paper uses fixed steps; this is the stated reading of a CFL.)
 */
fsp_status fsp_cfl_dt(const fsp_config* cfg, const fsp_block* blk, const double* metrics,
                      const void* Q, double cfl, double* dt_out, void* ws, size_t ws_bytes,
                      void* stream);

/*
 * fsp_norms -- per variable v: out[2v] = sqrt(mean over interior nodes of e^2),
 * out[2v+1] = max |e|, with e = A - B (B may be NULL: e = A).  out: 8 device doubles.
 * precision selects the element type of A and B.  Used for error norms and the
 * free-stream residual.
 */
fsp_status fsp_norms(const fsp_block* blk, int precision, const void* A, const void* B,
                     double* out, void* stream);

/*
 * fsp_check_state -- failure detection (the paper has no counterpart): *first_bad (one device
 * int64, written asynchronously on `stream`) receives the smallest linear index j ni + i of a
 * node whose state Q (state layout, cfg->precision) is not finite or not physical (rho <= 0 or
 * p <= 0, p = (gamma - 1)(E - |rho u|^2 / (2 rho))), or -1 when every node is valid.  The
 * caller reads it after the stream and maps a non-negative value to FSP_ERR_NONFINITE.
 * Argument errors: FSP_ERR_INVALID_ARG before anything is enqueued.
 */
fsp_status fsp_check_state(const fsp_config* cfg, const fsp_block* blk, const void* Q, long long* first_bad,
                           void* stream);

/*
 * ---- Discrete adjoint (FP64) --------------------------------------------------------
 * Vector-Jacobian products of the right-hand side, of one RK3 step and of the metrics, for
 * gradients of a scalar functional with respect to the state and the grid coordinates.
 * The paper has no adjoint; these are the exact reverse of the discrete operators above:
 * every nonlinear step of fsp_rhs (characteristic WENO with the mapped weights, the split
 * fluxes, the per-line maxima) is differentiated, so free-stream preservation carries into
 * the sensitivities.  At non-smooth points the derivative of |x| at 0 is +1, the mapping
 * branch is taken as in the forward pass, and the derivative of a line maximum goes to the
 * lowest index attaining it.  Adjoint outputs are accumulated (+=) into the caller's
 * buffers, which the caller zeroes.  The workspace must hold fsp_vjp_workspace_size bytes.
 * Every adjoint entry point, the size queries included, returns FSP_ERR_UNSUPPORTED for a
 * precision other than FSP_FP64 and for the options beyond the printed schemes (weights,
 * mid_split, scheme_alpha other than their defaults).
 */
fsp_status fsp_vjp_workspace_size(const fsp_config* cfg, const fsp_block* blk, size_t* bytes);

/* Q_bar += (d dQdt / dQ)^T dQdt_bar and metrics_bar += (d dQdt / dM)^T dQdt_bar over the
 * haloed metric array (metrics_bar nullable: the metric part is then discarded).  Ghost
 * contributions go back to the interior nodes they were formed from (periodic, transmissive,
 * slip wall with its normal, far field; Dirichlet ghosts carry none). */
fsp_status fsp_rhs_vjp(const fsp_config* cfg, const fsp_block* blk, const double* metrics,
                       const void* Q, const void* dQdt_bar, void* Q_bar, double* metrics_bar,
                       void* ws, size_t ws_bytes, void* stream);

/* Reverse of fsp_rk3_step at the step's input state Q_n: on entry Q_bar = dJ/dQ^{n+1}, on
 * return dJ/dQ^n; metrics_bar (nullable) += the step's metric adjoint.  The stages are
 * recomputed from Q_n (three right-hand sides, recorded in the workspace). */
fsp_status fsp_rk3_step_vjp(const fsp_config* cfg, const fsp_block* blk, const double* metrics,
                            const void* Q_n, double dt, void* Q_bar, double* metrics_bar, void* ws,
                            size_t ws_bytes, void* stream);

/* Recorded steps, for reverse sweeps over many steps.  A step tape (fsp_rk3_tape_size
 * bytes, device memory, 256-byte aligned, owned by the caller) holds the three stage states
 * Q^n, Q^(1), Q^(2) of one TVD-RK3 step (Section 6, Shu-Osher form), their right-hand sides
 * and their line maxima.  fsp_rk3_step_record advances Q in place by one step, as
 * fsp_rk3_step does (stage by stage, so the result may differ from it in the last bits),
 * and fills the tape; ws holds fsp_workspace_size bytes.  fsp_rk3_step_vjp_tape is the
 * reverse of that step read from its tape, with the argument meaning of fsp_rk3_step_vjp
 * and a workspace of fsp_vjp_workspace_size bytes; it runs no forward right-hand side. */
fsp_status fsp_rk3_tape_size(const fsp_config* cfg, const fsp_block* blk, size_t* bytes);
fsp_status fsp_rk3_step_record(const fsp_config* cfg, const fsp_block* blk, const double* metrics, void* Q,
                               double dt, void* tape, size_t tape_bytes, void* ws, size_t ws_bytes,
                               void* stream);
fsp_status fsp_rk3_step_vjp_tape(const fsp_config* cfg, const fsp_block* blk, const double* metrics,
                                 const void* tape, size_t tape_bytes, double dt, void* Q_bar,
                                 double* metrics_bar, void* ws, size_t ws_bytes, void* stream);

/* x_bar, y_bar += (d metrics / d(x, y))^T metrics_bar: the reverse of fsp_metrics through
 * the ghost-coordinate rule (periodic offsets are constants), with the scheme's own central
 * operator (scheme_alpha included). */
fsp_status fsp_metrics_vjp(const fsp_config* cfg, const fsp_block* blk, const double* x, const double* y,
                           const double* metrics_bar, double* x_bar, double* y_bar, void* stream);

/*
 * fsp_fma_peak -- throughput probe of the FP64 (precision FSP_FP64) or FP32 FMA pipe:
 * launches `blocks` x 256 threads, each running `iters` x 8 independent FMA chains, and
 * writes the chains' sum to sink[blocks * 256].  The floating-point operations done are
 * 2 * 8 * iters * blocks * 256.  Used to measure the ALU roof; no counterpart in the paper.
 */
fsp_status fsp_fma_peak(int precision, int blocks, int iters, void* sink, void* stream);

/*
 * fsp_round_to_float -- diagnostic of the FP32 paths' double-to-float rounding: for each of
 * the n doubles in[k] (device), out_int[k] receives the rounding done with integer operations
 * (the mixed path keeps its float-double conversions off the FP64 pipe) and out_hw[k] the
 * hardware conversion (round to nearest even).  They agree except that the integer rounding
 * flushes results below the float normal range to signed zero.  No counterpart in the paper.
 * FSP_ERR_INVALID_ARG for n < 0 or a pointer that is not device memory.
 */
fsp_status fsp_round_to_float(const double* in, float* out_int, float* out_hw, long long n, void* stream);

/*
 * fsp_widen_to_double -- diagnostic of the mixed path's float-to-double widening: for each of
 * the n floats in[k] (device), out_int[k] receives the widening done with integer operations
 * only and out_hw[k] the hardware conversion.  They agree bit for bit except that the integer
 * widening turns subnormals into signed zero (NaN stays NaN).  No counterpart in the paper.
 * FSP_ERR_INVALID_ARG for n < 0 or a pointer that is not device memory.
 */
fsp_status fsp_widen_to_double(const float* in, double* out_int, double* out_hw, long long n, void* stream);

/*
 * fsp_reciprocal_check -- diagnostic of the FP64 kernels' reciprocal and reciprocal square
 * root: for each of the n doubles in[k] (device), out (4 n doubles, device) receives at k the
 * reciprocal the kernels use (the hardware's approximate reciprocal refined by one third-order
 * Householder step), at n + k the correctly rounded 1/in[k], at 2 n + k the reciprocal square
 * root the kernels use (the hardware's approximation refined by one third-order step) and at
 * 3 n + k the IEEE 1/sqrt(in[k]) (two roundings); both square-root entries are 0 for
 * in[k] <= 0.  They agree to a few ulps for normal operands.  No counterpart in the paper.
 * FSP_ERR_INVALID_ARG for n < 0 or a pointer that is not device memory.
 */
fsp_status fsp_reciprocal_check(const double* in, double* out, long long n, void* stream);

/*
 * ---- Multi-block grids --------------------------------------------------------------
 * The paper's motivating case (Section 1): many structured blocks, of uneven sizes,
 * joined face to face.  The blocks partition the nodes of one larger grid: behind a face
 * of kind FSP_BC_LINK lie the linked block's own nodes, the ghost at depth k (k = 0 the
 * first) being the neighbour's node at depth k inward from its linked face, with the
 * index along the face running the same way or reversed.  Linked faces must match node
 * for node, and the neighbour must have at least 4 nodes across the face (state ghosts);
 * ghost coordinates follow links, periodic wraps or odd reflection through up to eight
 * layers, corners included.  Line maxima of the splitting are taken per block line.
 * The handle owns its device memory (descriptors, tile tables, per-block line maxima,
 * xi accumulators, RK stage states and, for FSP_FP64 and FSP_FP32_MIXED, the midpoint
 * metrics of every interface, for FSP_FP64 also the interfaces' characteristic directions and
 * the nodes' characteristic data that the xi pass leaves for the eta pass) from create to
 * destroy; no other call allocates.  The midpoint
 * metrics (the interpolation of Section 2.4) are taken from the bound metrics at the start of
 * each fsp_batch_rhs, fsp_batch_rk3_step and fsp_batch_tune, so the marching passes read them
 * instead of interpolating per right-hand side.
 * Each pass runs all blocks in one launch over a table of tiles (NL lines x T nodes, see
 * fsp_batch_tune); ghosts of linked faces are read straight from the neighbour's state,
 * so no halo copies are made.  Calls on one handle must not overlap.
 */
typedef struct {
  int nbr;            /* linked block (FSP_BC_LINK faces only)                         */
  int face;           /* its face, 0..3 (i-min, i-max, j-min, j-max)                   */
  int reversed;       /* 1: the index along the face runs the other way                */
  double offset[2];   /* added to coordinates across the link (periodic wraps)         */
} fsp_link;

typedef struct fsp_batch fsp_batch;

/* nblocks blocks (blocks[b].period used by their FSP_BC_PERIODIC faces), 4 face codes per
 * block in bc, 4 links per block in links (read for FSP_BC_LINK faces).  Shared settings
 * (scheme, precision, gamma, bc_state, ...) come from cfg.  *out receives the handle. */
fsp_status fsp_batch_create(const fsp_config* cfg, int nblocks, const fsp_block* blocks, const int* bc,
                            const fsp_link* links, fsp_batch** out);
/* Host arrays of nblocks device pointers: coordinates (nj*ni doubles), metrics
 * (fsp_metrics_elems doubles, written by fsp_batch_metrics) and the state of each block
 * (updated in place by fsp_batch_rk3_step).  Rebinding drops a captured graph. */
fsp_status fsp_batch_bind(fsp_batch* b, const double* const* x, const double* const* y,
                          double* const* metrics, void* const* Q);
/* fsp_metrics for every block, ghost coordinates through the links. */
fsp_status fsp_batch_metrics(fsp_batch* b, void* stream);
/* dQ/dt of every block (host array of device pointers, state layout). */
fsp_status fsp_batch_rhs(fsp_batch* b, void* const* dQdt, void* stream);
/* One direction (dir 0 = xi, 1 = eta) of every block, as fsp_flux_difference mode 0: the
 * difference H_{s+1/2} - H_{s-1/2} into D[b] (host array of device pointers; double for
 * FSP_FP64 and FSP_FP32_MIXED, float for FSP_FP32), for the bound states, with the line
 * maxima (and midpoint metrics) left by the last fsp_batch_rhs on this handle.  One launch
 * over all blocks. */
fsp_status fsp_batch_flux_difference(fsp_batch* b, int dir, void* const* D, void* stream);
/* One TVD-RK3 step of every block in lockstep; launches the captured graph when one was
 * captured for this dt. */
fsp_status fsp_batch_rk3_step(fsp_batch* b, double dt, void* stream);
/* fsp_batch_rk3_step end to end from host memory: copies each block's state from the host
 * array q_in[b] to the bound device state, takes one step as fsp_batch_rk3_step, and copies
 * the new state to q_out[b] (host arrays of nblocks host pointers, each 4*nj*ld elements in
 * the state layout and precision; q_in may equal q_out).  Blocks whose states lie the same
 * distance apart on the device and in both host arrays, under 512 bytes beyond each block's
 * end, are copied as one range including the padding between them, which the caller owns
 * on both sides.  Stream-ordered: q_out holds the result once the stream has completed (with
 * pageable host memory the copies also block the calling thread).  FSP_ERR_INVALID_ARG for
 * a null or device pointer or an unbound handle. */
fsp_status fsp_batch_rk3_step_host(fsp_batch* b, const void* const* q_in, void* const* q_out, double dt,
                                   void* stream);
/* Runs one step, then records one RK3 step (its kernels and memsets) as a CUDA graph that
 * later fsp_batch_rk3_step calls with the same dt launch as a whole.  The eager step
 * advances the state like any other step. */
fsp_status fsp_batch_capture_graph(fsp_batch* b, double dt, void* stream);

/* Tile shapes.  Variants 0-2 of a pass use 256-thread tiles of NL grid lines:
 *   xi  (dir 0): variant 0, 1, 2 = 2, 1, 4 lines of 128, 256, 64 interfaces;
 *   eta (dir 1): variant 0, 1, 2 = 8, 4, 16 lines of 32, 64, 16 interfaces.
 * xi variant 3 marches: each warp walks one row segment (rows longer than 512 nodes are cut
 * into equal segments) 32 nodes at a time, keeping the stencil nodes in a shared-memory
 * ring, with four rows per 128-thread CTA; fsp_batch_tile_shape reports 4 lines and 512
 * output nodes for it.  eta variant 3 marches too: a CTA of eight warps owns 32 adjacent
 * columns (one per lane) and walks a segment of them eight rows per step through a 16-row
 * shared-memory ring; fsp_batch_tile_shape reports 32 lines and the segment length.
 * Results do not depend on the variant (each interface is computed the same way); the
 * speed does.  Tiles are launched longest first, so that blocks of different sizes end the
 * pass with short tiles rather than a few long ones.  fsp_batch_tune picks, for each direction, the fastest variant on this
 * handle's blocks and bound state: it times five launches of each variant's pass (after two
 * untimed ones) with CUDA events on `stream` and waits for them.  With table_path non-null
 * it first looks up a key made of the device name and SM count, the scheme and arithmetic
 * options and a hash of the block sizes in that text file ("key vx ve ms_xi ms_eta" per
 * line, '#' comments; the last entry of a key wins).  If it finds the key it applies the
 * stored choice without timing; otherwise it times and appends the choice.  Changing a
 * shape synchronises the device and drops a captured graph (capture again after tuning).
 * Returns FSP_ERR_INVALID_ARG for an unbound handle or an unwritable table (the timed
 * choice is applied all the same).  The marching variants (3) are built for the default
 * options only (ppm = 1, linear_weights = 0, interp = 0): for other options the tuner skips
 * them and fsp_batch_set_tile_shape returns FSP_ERR_UNSUPPORTED for variant 3, leaving the
 * current variant.  fsp_batch_set_tile_shape forces a variant;
 * fsp_batch_tile_shape reports the current variant, lines per tile and output nodes per
 * line (any output pointer may be null). */
fsp_status fsp_batch_tune(fsp_batch* b, const char* table_path, void* stream);
fsp_status fsp_batch_set_tile_shape(fsp_batch* b, int dir, int variant);
fsp_status fsp_batch_tile_shape(const fsp_batch* b, int dir, int* variant, int* lines, int* outputs);
fsp_status fsp_batch_destroy(fsp_batch* b);

/* ---- three dimensions (Sections 2.1-2.2) ------------------------------------------------
 * Q = (rho, rho u, rho v, rho w, e) with e = p/(gamma - 1) + rho |u|^2 / 2 (Eq. 2.1), on one
 * block of ni x nj x nk nodes.  Layouts (device memory, caller-owned): coordinates x, y, z
 * [nk][nj][ni] doubles; state [5][nk][nj][ni] doubles (i fastest, no row padding); metrics
 * fsp3_metrics_elems() doubles, 10 planes on the node range extended by FSP_G layers:
 * plane 3 d + c is component c (x, y, z) of the metric of direction d (xi, eta, zeta), i.e.
 * xi_x^, xi_y^, xi_z^, eta_x^, ..., zeta_z^, and plane 9 is J^-1; node (i, j, k) of plane p
 * at p P + ((k + G)(nj + 2G) + (j + G))(ni + 2G) + (i + G), P = (ni+2G)(nj+2G)(nk+2G).
 * FP64 only and the printed schemes' options only (cfg->precision FSP_FP64, weights,
 * mid_split and scheme_alpha at their defaults), else FSP_ERR_UNSUPPORTED; cfg->bc is not
 * used.  Faces FSP_BC_PERIODIC or FSP_BC_TRANSMISSIVE (others: FSP_ERR_UNSUPPORTED), both
 * faces of a direction periodic or neither, and a non-periodic direction needs >= 13 nodes
 * (FSP_ERR_INVALID_ARG otherwise).  Ghost states: periodic wrap or a copy of the boundary
 * node; ghost coordinates: periodic wrap plus the period vector, else odd reflection about
 * the boundary node.  Host pointers and short workspaces give FSP_ERR_INVALID_ARG.  No
 * adjoint. */
typedef struct fsp3_block {
  int ni, nj, nk;
  int bc[6];               /* faces i-min, i-max, j-min, j-max, k-min, k-max */
  double period[3][3];     /* (dx, dy, dz) added per periodic wrap in i, j and k */
} fsp3_block;

/* Doubles of the metric array (10 planes on the extended node range). */
long long fsp3_metrics_elems(const fsp3_block* blk);

/* Bytes of workspace for every fsp3_* call (the largest of the metric scratch and the RK3
 * step's line maxima, accumulator and two stage states). */
fsp_status fsp3_workspace_size(const fsp_config* cfg, const fsp3_block* blk, size_t* bytes);

/* fsp3_metrics -- the symmetric conservative metrics of Eq. 2.4,
 *   m_{d,c} = 1/2 [(p_a q)_b - (p_b q)_a + (q_b p)_a - (q_a p)_b],
 * (a, b) the directions after d and (p, q) the coordinates after c, cyclically (for xi_x^
 * this is Eq. 2.4 as printed), and J^-1 = 1/3 sum_{d,c} m_{d,c} (c)_d (Eq. 2.5).  Every
 * derivative, inner and outer, is the scheme's central operator delta^{c,(1)} (Eq. 2.7)
 * with the midpoint interpolation of cfg->interp, so that the metric identities hold to
 * round-off and a uniform flow is preserved on any grid. */
fsp_status fsp3_metrics(const fsp_config* cfg, const fsp3_block* blk, const double* x, const double* y,
                        const double* z, double* metrics, void* ws, size_t ws_bytes, void* stream);

/* Line maxima of |U^| + c|k^| (without the factor lf_alpha) into lam: the xi lines
 * [nk][nj], then the eta lines [nk][ni], then the zeta lines [nj][ni]. */
fsp_status fsp3_line_lambda(const fsp_config* cfg, const fsp3_block* blk, const double* metrics, const double* Q,
                            double* lam, void* stream);

/* fsp3_rhs -- dQ/dt = -(dE^/dxi + dF^/deta + dG^/dzeta) / J^-1 (Eq. 2.2), each direction
 * with the splitting of Section 2.3 and the upwind-biased combination of Section 3; the
 * characteristic projection uses the direction n of the averaged metrics and, for the
 * eigenspace of Un, the entropy wave and two shear waves along t1 = a x n / |a x n| (a the
 * coordinate axis least aligned with n, ties to the later axis) and t2 = n x t1. */
fsp_status fsp3_rhs(const fsp_config* cfg, const fsp3_block* blk, const double* metrics, const double* Q,
                    double* dQdt, void* ws, size_t ws_bytes, void* stream);

/* fsp3_rk3_step -- one TVD-RK3 step of size dt, Q updated in place. */
fsp_status fsp3_rk3_step(const fsp_config* cfg, const fsp3_block* blk, const double* metrics, double* Q, double dt,
                         void* ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FSP_H */
