/*
 * fsei.h -- C ABI of libfsei.so: one time step of the second-order,
 * staggered-grid, fractional-step Navier-Stokes integrator of the FSEI
 * cardiac solver (arXiv 2103.15187), as hand-written CUDA for sm_103a.
 *
 * Method (Sec. 2.1, Eq. 2-3; Sec. 3.1):
 *   * incompressible Navier-Stokes, non-dimensional, Newtonian stress
 *     tau = 2 Re^-1 E (Sec. 2.1), body force f given per step (the immersed
 *     boundary forcing enters the fractional step as this field, Sec. 3.2);
 *   * central second-order differences on a staggered mesh (Sec. 2.1);
 *   * Adams-Bashforth for advection, Crank-Nicolson for viscosity,
 *     gamma = 3/2, rho = -1/2 (Eq. 3); first step of a run: gamma = 1,
 *     rho = 0 (no H^{n-1} yet);
 *   * fractional step: predictor with the old pressure, pressure-increment
 *     Poisson equation, projection, p^{n+1} = p^n + phi - beta L phi with
 *     beta = dt / (2 Re);
 *   * the implicit viscous operator approximately factorised into one
 *     tridiagonal system per direction, periodic x and y handled as cyclic
 *     systems (Sec. 3.1);
 *   * periodic x, y; z either periodic (uniform) or bounded by no-slip walls
 *     at z = -1, +1 with a tanh-stretched mesh (Sec. 4, Sec. 5).
 *
 * Field layout (all fields): contiguous row-major [nz][ny][nx], x fastest,
 * element type double (FSEI_FP64) or float (FSEI_MIXED).  Staggering:
 *   u at (x_i, y_{j+1/2}, zc_k), v at (x_{i+1/2}, y_j, zc_k),
 *   w at (x_{i+1/2}, y_{j+1/2}, z_k), p at (x_{i+1/2}, y_{j+1/2}, zc_k),
 * x_i = i lx/nx, y_j = j ly/ny, z_k the z faces, zc_k = (z_k + z_{k+1})/2.
 * With walls w[k=0] is the bottom wall face and must hold 0; the top wall
 * face is not stored.
 *
 * Ownership: the caller owns every field buffer (device memory, 16-byte
 * aligned).  The library owns its workspace, plans and z metrics, allocated
 * in fsei_grid_create and freed by fsei_grid_destroy.
 *
 * Errors: no entry point throws or aborts.  Argument, shape and alignment
 * errors are reported at call time; asynchronous conditions found on the
 * device (non-finite values, CFL number above 1) are reported through
 * fsei_step_stats.flags and the status of a call that synchronises (one that
 * asks for stats).  fsei_last_error() gives a message for the last non-OK
 * status of the calling thread.
 *
 * Concurrency: a grid handle is not re-entrant; calls are ordered on the
 * CUDA stream passed in (NULL = legacy default stream).
 */
#ifndef FSEI_H
#define FSEI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FSEI_OK = 0,
    FSEI_E_ARG = 1,         /* NULL handle/pointer, bad parameter value      */
    FSEI_E_SHAPE = 2,       /* unsupported extent (see fsei_grid_create)     */
    FSEI_E_UNSUPPORTED = 3, /* valid request this build does not implement   */
    FSEI_E_NOMEM = 4,       /* device allocation failed                      */
    FSEI_E_CUDA = 5,        /* a CUDA runtime call failed                    */
    FSEI_E_NONFINITE = 6,   /* a NaN/Inf appeared in the new state           */
    FSEI_E_CFL = 7,         /* CFL number of the new state above 1           */
    FSEI_E_BOUNDS = 8       /* bounds-checking mode: a kernel wrote outside a
                               workspace buffer (fsei_grid_check_bounds)     */
} fsei_status;

typedef enum {
    FSEI_FP64 = 0,  /* every stored value and every operation in double      */
    FSEI_MIXED = 1  /* float fields, stencils, FFTs and sweeps; double for the
                       zero and near-zero wavenumber Poisson systems and for
                       all global reductions (dt, CFL, divergence, energy)  */
} fsei_precision;

typedef enum { FSEI_Z_PERIODIC = 0, FSEI_Z_WALLS = 1 } fsei_zbc;

/* Step-statistics flags (bit set in fsei_step_stats.flags). */
#define FSEI_FLAG_NONFINITE 1
#define FSEI_FLAG_CFL 2

typedef struct {
    int32_t nx, ny, nz;     /* cells; nx, ny even, of the form 2^a 3^b,
                               nx/2 >= 4, ny >= 4, 8 <= nz <= 2048; nx/2
                               and ny at most 1024 */
    double lx, ly;          /* periodic box lengths in x and y */
    int32_t zbc;            /* fsei_zbc */
    double lz;              /* periodic z: box length (uniform mesh);
                               walls: ignored, z spans [-1, 1] */
    double stretch;         /* walls: tanh clustering factor s,
                               z_k = tanh(s (2k/nz - 1)) / tanh(s);
                               0 = uniform */
    const double *zfaces;   /* optional host array of nz+1 increasing z
                               faces (walls only); overrides stretch */
    int32_t prec;           /* fsei_precision */
    double near_zero_tau;   /* FSEI_MIXED: a Poisson mode (kx, ky) is solved
                               in double when (lambda_x + lambda_y) Lz^2 <
                               tau, lambda the modified wavenumbers
                               (2 - 2 cos(2 pi k / n)) / h^2, Lz the z
                               extent; <= 0 selects 64 */
} fsei_grid_desc;

typedef struct fsei_grid_s *fsei_grid;

/* Device pointers to caller-owned fields (element type per precision).
 * hu, hv, hw hold the advection term H^{n-1} of the previous step on input
 * and H^n on output (Eq. 3's Adams-Bashforth history).  have_prev_h = 0
 * makes the first step of the call use gamma = 1, rho = 0; the library sets
 * it to 1 on return. */
typedef struct {
    void *u, *v, *w, *p, *hu, *hv, *hw;
    int32_t have_prev_h;
} fsei_state;

/* Time-integration scheme of fsei_step_params.scheme (Sec. 2.1).
 *   FSEI_AB2_CN: Eq. 3, Adams-Bashforth advection with weights gamma, rho,
 *     Crank-Nicolson viscosity, one fractional step per time step;
 *   FSEI_RK3_CN: the third-order Runge-Kutta variant the paper notes beside
 *     it (low-storage scheme of its cited Rai & Moin / Verzicco & Orlandi):
 *     three fractional sub-steps l = 1, 2, 3 with advection weights
 *     gamma_l = 8/15, 5/12, 3/4 and rho_l = 0, -17/60, -5/12 (previous
 *     sub-step), viscous, pressure and force terms over alpha_l dt with
 *     alpha_l = gamma_l + rho_l, Crank-Nicolson within each sub-step.
 *     params->gamma and ->rho are not used; dt (or the CFL rule on u^n) is
 *     the full step's; H of the last sub-step is stored as the history. */
typedef enum { FSEI_AB2_CN = 0, FSEI_RK3_CN = 1 } fsei_scheme;

/* Constitutive law of fsei_step_params.rheology (Sec. 2.1).
 *   FSEI_NEWTONIAN: tau = 2 Re^-1 E;
 *   FSEI_CARREAU_YASUDA: shear-thinning blood, tau = 2 Re^-1 eta(gdot) E
 *     with eta = eta_inf + (1 - eta_inf) (1 + (lambda gdot)^a)^((n - 1) / a)
 *     relative to the zero-shear viscosity (Re built on it), gdot =
 *     sqrt(2 E:E).  The Newtonian part stays in the implicit Crank-Nicolson
 *     sweeps; the remainder div(2 Re^-1 (eta - 1) E) of u^n is explicit and
 *     joins the advection term H (same Adams-Bashforth weights, stored in
 *     the history).  Strain rates at the centres and at the advection's
 *     edge points, gdot at the centres, the excess viscosity averaged back
 *     to the edges.  Adams-Bashforth scheme only. */
typedef enum { FSEI_NEWTONIAN = 0, FSEI_CARREAU_YASUDA = 1 } fsei_rheology;
typedef struct {
    double lambda;     /* time constant (in the flow's time unit), >= 0 */
    double n;          /* power-law index, > 0 */
    double a;          /* Yasuda exponent, > 0 */
    double eta_inf;    /* infinite-shear viscosity over the zero-shear one, in [0, 1] */
} fsei_carreau_yasuda;

typedef struct {
    double re;          /* Reynolds number (> 0) */
    double dt;          /* time step when cfl <= 0 */
    double cfl;         /* > 0: dt = cfl / max_cells(|u_c|/dx + |v_c|/dy +
                           |w_c|/dz_k) recomputed on the device from u^n
                           every step (u_c, v_c, w_c: two-face averages at
                           the cell centre) */
    double gamma, rho;  /* Adams-Bashforth weights, normally 1.5, -0.5 */
    double fconst[3];   /* uniform body force added to f (e.g. a channel's
                           pressure-gradient drive 2/Re in x) */
    int32_t scheme;     /* fsei_scheme (0: Adams-Bashforth, Eq. 3) */
    int32_t rheology;   /* fsei_rheology (0: Newtonian) */
    fsei_carreau_yasuda cy;   /* FSEI_CARREAU_YASUDA parameters */
} fsei_step_params;

typedef struct {
    double dt_used;        /* dt of the last step (the full step's dt) */
    double cfl;            /* dt_used * max_cells(...) of the new state */
    double max_div;        /* max over cells of |D u^{n+1}| */
    double kinetic_energy; /* 1/2 sum u^2 dV over all staggered points */
    int32_t flags;         /* FSEI_FLAG_* */
} fsei_step_stats;

/* Create a grid handle: z metrics, plans and workspace on the current CUDA
 * device.  Returns FSEI_E_SHAPE for unsupported extents, FSEI_E_ARG for bad
 * lengths or faces, FSEI_E_NOMEM if the workspace does not fit.  When the
 * environment variable FSEI_WORKSPACE_LIMIT_BYTES holds a decimal number at
 * the call, the handle's device allocations may not exceed that many bytes
 * in total; a grid that needs more fails with FSEI_E_NOMEM (a memory budget
 * for a process that shares the GPU).  When FSEI_CHECK_BOUNDS is set to a
 * value other than "0" at the call, the grid runs in bounds-checking mode
 * (see fsei_grid_check_bounds). */
fsei_status fsei_grid_create(const fsei_grid_desc *desc, fsei_grid *out);

/* Release a handle (NULL is a no-op).  Synchronises the device first. */
void fsei_grid_destroy(fsei_grid grid);

/* Bytes of device workspace the handle owns. */
int64_t fsei_grid_workspace_bytes(fsei_grid grid);

/* Launch schedule of a grid: the tile shapes and solver splits its tunable
 * kernels run with.  The paper fixes none of them (its Sec. 3 maps the same
 * sweeps and transforms onto its own GPUs); every admissible value computes
 * the same quantities with the same operations grouped differently, so
 * results agree to rounding and only the time changes.  0 marks a field
 * whose kernel does not apply to the grid's extents.
 *   rhs_cells_per_lane: RHS + x sweep (Eq. 3, Sec. 3.1), cells of a grid row
 *     per lane of the row-resident kernel (4, or 2 or 8 in FSEI_MIXED);
 *   rhs_rows_per_strip: 0 for one grid row per lane; 4, 8 or 16 (where ny
 *     allows) for lanes that march that many consecutive rows of a plane,
 *     reusing the stencil rows two neighbours share and fetching the next
 *     row's while computing one (16 or 32 bytes per lane, 16 to 128 lanes
 *     per row);
 *   poisson_lanes_per_line, poisson_rows_per_lane: z tridiagonal solve of
 *     each Fourier mode of the pressure equation (Sec. 2.1; Sec. 3.1 and
 *     Sec. 4 on its parallel solve): lanes that share a line (reduction
 *     across lanes) and rows each lane eliminates on its own; their product
 *     is nz;
 *   rfft_rows_per_block: forward x transform, grid rows per thread block;
 *   ffty_columns_per_block: y transforms, kx columns per thread block;
 *   project_passes_per_thread: projection and pressure update (Eq. 3),
 *     row passes per thread;
 *   zsweep_columns_per_lane: z sweep (Sec. 3.1), x columns each lane
 *     solves (1, or 2 with one chunk's factors read once for both, where
 *     the z lines split into chunks of at most 16 rows). */
typedef struct {
    int32_t rhs_cells_per_lane;
    int32_t poisson_lanes_per_line;
    int32_t poisson_rows_per_lane;
    int32_t rfft_rows_per_block;
    int32_t ffty_columns_per_block;
    int32_t project_passes_per_thread;
    int32_t rhs_rows_per_strip;
    int32_t zsweep_columns_per_lane;
} fsei_schedule;

/* fsei_grid_autotune flag: measure again although this process already
 * holds a schedule for the grid's shape. */
#define FSEI_TUNE_FORCE 1

/* Pick the grid's schedule by measurement.  For each field in turn, the
 * others held, every admissible value runs inside whole fractional steps
 * (one untimed, eight timed) on stand-in fields of the grid's extents that
 * the call allocates (7 fields) and frees; CUDA events around the kernel
 * that the field shapes give its device time, and the value of least time
 * is kept (a challenger must be 1% faster than the value in place).  The
 * choice is applied to the grid and remembered for the process under the
 * grid's (device, precision, nx, ny, nz, zbc): every grid created later
 * with that key, and a later autotune call without FSEI_TUNE_FORCE, takes
 * it without measuring, so grids of one shape run identical kernels.
 * Synchronises the device; allocates; not allowed inside a stream capture.
 * The grid's per-kernel timing sums and step scalars are left as they were;
 * no caller field is touched.  out (optional) receives the schedule.
 * Returns FSEI_E_NOMEM when the stand-in fields do not fit, FSEI_E_ARG for
 * a NULL grid or unknown flags, FSEI_E_CUDA if a launch fails. */
fsei_status fsei_grid_autotune(fsei_grid grid, int32_t flags, void *cuda_stream,
                               fsei_schedule *out);

/* The schedule the grid runs with now. */
fsei_status fsei_grid_get_schedule(fsei_grid grid, fsei_schedule *out);

/* Run the grid with the given schedule (e.g. one recorded by an earlier
 * autotune, for runs that must repeat bit for bit).  FSEI_E_ARG if a field
 * is not admissible for the grid (0 is admissible exactly where the kernel
 * does not apply).  Takes effect at the next launch; not remembered for
 * other grids. */
fsei_status fsei_grid_set_schedule(fsei_grid grid, const fsei_schedule *in);

/* Advance the state by nsteps fractional steps (Eq. 3 with the
 * approximate factorisation of Sec. 3.1).  fx, fy, fz: body force at the u,
 * v and w points, constant over the call, or NULL for zero.  out: if not
 * NULL, the call synchronises the stream and fills the statistics of the
 * last step; its status then reports device flags (FSEI_E_NONFINITE first,
 * then FSEI_E_CFL).  Without out the call is asynchronous. */
fsei_status fsei_step(fsei_grid grid, fsei_state *state, const void *fx,
                      const void *fy, const void *fz,
                      const fsei_step_params *params, int32_t nsteps,
                      void *cuda_stream, fsei_step_stats *out);

/* fsei_step on a state held in host memory: the seven fields of `host` are
 * copied into the device buffers of `dev`, nsteps steps run on them exactly
 * as fsei_step would run them (the same kernels, the same results), and the
 * seven fields are copied back into `host`.  host->have_prev_h plays the
 * role of state->have_prev_h (dev->have_prev_h is ignored).
 *   host: nx*ny*nz values of the grid's precision per field (pinned memory,
 *     cudaHostAlloc or cudaHostRegister, for asynchronous copies; pageable
 *     memory works, with copies that block the calling thread);
 *   dev: caller-owned device buffers of the same sizes, 16-byte aligned,
 *     used as the step's state; every field is overwritten by the copy in.
 * Ordering: the copies in wait for the work queued on cuda_stream before
 * the call and, field by field, for that field's copy back from the
 * previous fsei_step_host call on this grid; the steps wait for the copies
 * in.  The copies back run on the grid's own copy stream: the history
 * fields H^n as soon as the last step's right-hand side has written them
 * (under the rest of that step), u, v, w, p after the step; they are not
 * ordered before work queued on cuda_stream after the call unless out is
 * given or fsei_step_host_join is called.  Neither `host` nor `dev` may be
 * touched by other work until then.  out: as in fsei_step (the call then
 * also waits for the copies back).  Errors as fsei_step; FSEI_E_ARG for
 * NULL fields or a misaligned device field. */
fsei_status fsei_step_host(fsei_grid grid, fsei_state *host, const fsei_state *dev,
                           const void *fx, const void *fy, const void *fz,
                           const fsei_step_params *params, int32_t nsteps,
                           void *cuda_stream, fsei_step_stats *out);

/* Order the work queued on cuda_stream after this call behind the copies
 * back of the last fsei_step_host call on the grid (no-op before the first
 * such call).  Synchronising cuda_stream afterwards makes the host fields
 * complete. */
fsei_status fsei_step_host_join(fsei_grid grid, void *cuda_stream);

/* Pressure-increment Poisson solve of the fractional step (Sec. 2.1: the
 * elliptic equation whose solution makes u^{n+1} solenoidal; Sec. 4: solved
 * with transforms in the two periodic directions): phi with
 * D G phi = rhs at the cell centres (D G: the compound staggered Laplacian,
 * Neumann at walls), phi of zero volume-weighted mean.  rhs must have zero
 * volume-weighted mean (sum rhs dz_k = 0) -- the solve pins phi at k = 0 of
 * the (0, 0) Fourier mode and leaves that row to compatibility.  rhs and
 * phi: device fields of the grid's element type; they may alias. */
fsei_status fsei_poisson_solve(fsei_grid grid, const void *rhs, void *phi,
                               void *cuda_stream);

/* Discrete adjoint of one step: the exact transpose (Euclidean inner product
 * of the stored arrays) of the step's map (u^n, p^n, H^{n-1}, f) ->
 * (u^{n+1}, p^{n+1}, H^n) at a frozen dt (Eq. 3 with the factorisation of
 * Sec. 3.1; the CFL maximum is not differentiable, so params->cfl must be
 * <= 0 and params->dt the step's dt).
 *   fwd:  the step's inputs; u, v, w read (p and H are not needed: the step
 *         is linear in them), have_prev_h selects gamma, rho as in fsei_step.
 *   adj:  in: cotangents of the outputs u, v, w, p (step n+1) and hu, hv, hw
 *         (the stored H^n); out, in place: cotangents of the inputs u, v, w,
 *         p (step n) and hu, hv, hw (H^{n-1}).
 *   fbar_x/y/z: if not NULL, the cotangent of the body force is added.
 * With walls the wall face w[0] is not an input: its cotangent is 0.  The
 * first call allocates three fields of adjoint workspace.  Asynchronous. */
fsei_status fsei_adjoint_step(fsei_grid grid, const fsei_state *fwd,
                              const fsei_step_params *params, fsei_state *adj,
                              void *fbar_x, void *fbar_y, void *fbar_z,
                              void *cuda_stream);

/* Immersed-boundary forcing (Sec. 2.1, Eq. 4; Sec. 3.2): the no-slip
 * condition of a moving surface imposed on Lagrangian markers (the
 * centroids of its triangles).  For every marker b and velocity component,
 * the 3 x 3 x 3 nodes of that component's staggered grid nearest to x_b form
 * its support; the transfer operators phi_k of a moving-least-squares fit
 * (linear basis [1, x, y, z], weight exp(-r^2) with r the node offset over
 * the nearest node's control extents dx, dy and dz_k (centre points) or
 * hc_k (w faces)) interpolate the field, u(x_b) = sum_k phi_k u_k; the
 * direct force F_b = (U_b - u(x_b)) / dt is spread back over the same nodes,
 * f_k += phi_k F_b dV_b / dV_k (dV_k = dx dy dz_k, or dx dy hc_k for w), so
 * that sum(f dV) = sum(F dV_b).  The fits run in double.
 *   u, v, w: the velocity to interpolate (device fields of the grid's type);
 *   xb, ub: device arrays of nmarkers x 3 doubles (positions, prescribed
 *     velocities); dvb: nmarkers forcing volumes (e.g. face area times the
 *     local cell size);
 *   fx, fy, fz: device fields the force is added to (atomically; the sum
 *     over markers does not depend on their order beyond rounding);
 *   u_at: NULL or device nmarkers x 3 doubles, the interpolated velocity.
 * A marker whose support would leave the interior z nodes of a walled grid
 * (within about one cell of a wall) is skipped; with skipped != NULL the
 * call synchronises and writes their count.  Positions outside the periodic
 * box are wrapped.  FSEI_E_ARG for NULL fields, bad counts or dt <= 0. */
fsei_status fsei_ib_forcing(fsei_grid grid, const void *u, const void *v, const void *w,
                            const double *xb, const double *ub, const double *dvb,
                            int32_t nmarkers, double dt, void *fx, void *fy, void *fz,
                            double *u_at, void *cuda_stream, int32_t *skipped);

/* Hydrodynamic loads on the wet faces (Sec. 2.1, Eqs. 5-7): the pressure
 * and the viscous stress tau = Re^-1 (grad u + grad u^T) at the probe point
 * x_f + probe n_f off each face, from the fits above (the gradient is the
 * fit's linear coefficients); face load F_f = (-p n_f + tau . n_f) A_f
 * (Eq. 6), for a two-sided face (valve leaflet) minus the same at
 * x_f - probe n_f (Eq. 5); a third of F_f is added to each of the face's
 * three nodes (Eq. 7).
 *   p, u, v, w: device fields of the grid's type;
 *   xf, nf: device nfaces x 3 doubles (centroids, unit normals pointing into
 *     the fluid on the + side); af: nfaces areas; two_sided: NULL (all
 *     one-sided) or nfaces flags;
 *   face_force: device nfaces x 3 doubles, written;
 *   tris, node_force: NULL, or nfaces x 3 node indices and nnodes x 3
 *     doubles the nodal loads are added to.
 * Faces whose probe support leaves the interior get zero load and are
 * counted in skipped[0]; node indices outside [0, nnodes) are counted in
 * skipped[1] (skipped: NULL or 2 ints; the call then synchronises). */
fsei_status fsei_ib_loads(fsei_grid grid, const void *p, const void *u, const void *v,
                          const void *w, const double *xf, const double *nf, const double *af,
                          const int32_t *two_sided, const int32_t *tris, int32_t nfaces,
                          int32_t nnodes, double probe, double re, double *face_force,
                          double *node_force, void *cuda_stream, int32_t *skipped);

/* Batched ensemble of independent boxes of uneven sizes (each with its own
 * grid description, Reynolds number, dt or CFL, body force and state).
 * fsei_batch_create creates one grid per box (as fsei_grid_create) plus the
 * streams and events of a CUDA graph.  fsei_batch_step advances every box by
 * nsteps fractional steps.  Boxes with the same description and launch
 * schedule form a group: each pass of the step is one kernel launch over all
 * boxes of the group (the box in blockIdx.z, its arguments from a table
 * passed with the launch).  One step of all groups is captured into a CUDA
 * graph, groups on parallel branches, and the graph is replayed once per
 * step on cuda_stream.  The graph is re-captured when
 * the state pointers, forces, parameters or history flags differ from the
 * last capture (the first call, and the call after it, capture).
 *   states: nboxes fsei_state (device pointers per box, have_prev_h updated);
 *   forces: NULL, or 3*nboxes pointers (fx, fy, fz per box, each nullable);
 *   params: nboxes fsei_step_params;
 *   out: NULL or nboxes fsei_step_stats (the call then synchronises; the
 *        status reports the first box with a device flag).
 * Each box's results agree with fsei_step on that box alone to rounding
 * (the grouped launches run the same kernel bodies from another entry
 * point, so the last bits may differ). */
typedef struct fsei_batch_s *fsei_batch;
fsei_status fsei_batch_create(const fsei_grid_desc *descs, int32_t nboxes,
                              fsei_batch *out);
void fsei_batch_destroy(fsei_batch batch);
int32_t fsei_batch_size(fsei_batch batch);
/* Boxes per launch group (default 0: no limit): the boxes of one group
 * (same description and schedule) are split into launch groups of at most
 * max_boxes, each with its own kernel launches, spread over the graph's
 * parallel branches.  Larger groups launch fewer, larger kernels; smaller
 * ones let different passes of different groups run side by side.  Drops
 * the captured graphs.  FSEI_E_ARG for a NULL batch or max_boxes < 0. */
fsei_status fsei_batch_set_max_group(fsei_batch batch, int32_t max_boxes);
/* Launch groups of the last captured graph (0 before the first capture). */
int32_t fsei_batch_launch_groups(fsei_batch batch);
/* fsei_grid_autotune for every box (one measurement per distinct shape;
 * flags as there), then, for each description shared by two or more boxes,
 * a second pass timed as that group's launches: knob by knob, every
 * admissible value applied to all of the group's boxes, one step of the
 * group captured into a graph on stand-in fields (7 per box, allocated and
 * freed by the call; the pass is skipped for a group whose stand-ins do not
 * fit) and replayed seven times; the value of least median time is kept (a
 * challenger must be 0.5 % faster) and remembered for the shape as
 * fsei_grid_autotune remembers its choice; a group of the same shape and
 * box count is measured once per process unless flags has
 * FSEI_TUNE_FORCE.  Synchronises the device.
 * Drops the captured graphs, which the next fsei_batch_step captures again
 * with the new schedules. */
fsei_status fsei_batch_autotune(fsei_batch batch, int32_t flags, void *cuda_stream);
fsei_status fsei_batch_step(fsei_batch batch, fsei_state *states,
                            const void *const *forces,
                            const fsei_step_params *params, int32_t nsteps,
                            void *cuda_stream, fsei_step_stats *out);

/* Size in bytes of the device array that backs fsei_poisson_solve_noalloc. */
#define FSEI_NOALLOC_SCRATCH_BYTES (32u << 20)

/* Allocation-free Poisson solve.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they need
 * a solve -- a host application that owns every allocation and hands the
 * library raw pointers only, code whose device memory is already fully
 * reserved by a caching allocator, or loops that must not pay the implicit
 * synchronisation of cudaMalloc/cudaFree.  It computes the same phi as
 * fsei_poisson_solve for a grid described by desc, without a grid handle:
 * all scratch (metrics, twiddles, wavenumber tables, spectrum) lives in one
 * file-scope device array of FSEI_NOALLOC_SCRATCH_BYTES (32 MiB) that every
 * GPU loading the library holds until the process exits.  It calls no
 * cudaMalloc/cudaFree and no allocating routine, on the device or the host.
 *   desc: as for fsei_grid_create (zfaces read during the call only);
 *   rhs, phi: device fields [nz][ny][nx] of the precision's element type,
 *   16-byte aligned, caller-owned; rhs with zero volume-weighted mean.
 * Returns FSEI_E_SHAPE when the extents are unsupported or the grid needs
 * more scratch than the array holds (e.g. FP64 up to about 128^3 cells),
 * FSEI_E_ARG for bad arguments, FSEI_E_CUDA if a CUDA call fails.  It does
 * not set fsei_last_error().  The first call on a device (made with that
 * device current) looks up the array's device address.  A call on a stream
 * that is being captured is refused with FSEI_E_ARG (a captured copy would
 * read the static host buffer at replay, after later calls have rewritten
 * it).  All calls share the array, which keeps the
 * last call's contents (the spectrum is cleared on every call); calls whose
 * GPU work overlaps -- on different streams or from different host
 * threads -- race on it and must be serialised by the caller.  The tables
 * are built in a static host buffer and copied from it on the given stream;
 * the call returns once that buffer may be reused by the next call. */
fsei_status fsei_poisson_solve_noalloc(const fsei_grid_desc *desc,
                                       const void *rhs, void *phi,
                                       void *cuda_stream);

/* Bounds-checking mode, a debugging aid with no counterpart in the paper
 * (it stands in for a memory checker where none can run).  A grid created
 * with FSEI_CHECK_BOUNDS set places a guard zone before and after every
 * buffer of its workspace (1/16 of the buffer, at least 64 KiB, at most
 * 1 MiB), filled with all-ones bytes for floating-point buffers (a NaN: a
 * kernel that reads a guard makes its results non-finite, which the step
 * flags as FSEI_E_NONFINITE) and zero bytes for integer ones.  This call
 * synchronises the device and returns FSEI_E_BOUNDS, with the buffer, side
 * and distance in fsei_last_error(), if any guard byte changed (a write past
 * the end of a buffer), FSEI_OK otherwise; FSEI_E_UNSUPPORTED for a grid
 * created without the mode.  In the mode, fsei_step, fsei_step_host,
 * fsei_poisson_solve, fsei_adjoint_step, fsei_ib_forcing, fsei_ib_loads and
 * fsei_batch_step (every box) run this check before they return, so they
 * synchronise.  The caller's own fields are not guarded. */
fsei_status fsei_grid_check_bounds(fsei_grid grid);

/* Test hook of the bounds-checking mode (no counterpart in the paper):
 * changes the guard byte `offset` bytes from the edge of workspace buffer
 * `buffer` (allocation order), before it (side 0) or after it (side 1), so
 * that a test can check that fsei_grid_check_bounds reports the write.  The
 * byte lies inside the library's own allocation.  Synchronises the device.
 * FSEI_E_UNSUPPORTED without the mode, FSEI_E_ARG for a zone or offset that
 * does not exist. */
fsei_status fsei_grid_poke_guard(fsei_grid grid, int32_t buffer, int32_t side, int64_t offset);

/* Per-kernel timing, for measurement tools.  While enabled, fsei_step and
 * fsei_poisson_solve record a CUDA event pair on the call's stream around
 * every kernel they launch.  fsei_kernel_times synchronises the device,
 * writes for each kernel kind k < cap the summed device time in ms and the
 * number of launches since the last call, resets the sums, and returns the
 * number of kinds.  fsei_kernel_name(k) names kind k (NULL if out of range).
 * Timing does not change what the kernels compute. */
fsei_status fsei_set_kernel_timing(fsei_grid grid, int32_t enable);
int32_t fsei_kernel_times(fsei_grid grid, double *total_ms, int64_t *launches,
                          int32_t cap);
const char *fsei_kernel_name(int32_t kind);

/* Measurement helper (the paper has no counterpart): the current device's
 * double-precision fused multiply-add throughput, in 10^9 thread
 * instructions per second -- the best of three timed launches of a kernel
 * that fills every SM with independent DFMA chains.  The FP64 step is bound
 * by this pipe, so measurement tools use the figure as its arithmetic peak.
 * Synchronises the stream; FSEI_E_CUDA if a launch fails. */
fsei_status fsei_fp64_fma_rate(void *cuda_stream, double *ginst_per_s);

/* Message for the calling thread's last non-OK status ("" if none). */
const char *fsei_last_error(void);

/* Library version string. */
const char *fsei_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FSEI_H */
