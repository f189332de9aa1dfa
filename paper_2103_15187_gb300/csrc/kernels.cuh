// Launch interface between the host library (api.cu) and the kernels of one
// fractional step.  Internal to libfsei.so.
#pragma once
#include <string.h>

#include <cuda/std/tuple>
#include <utility>
#include <vector>

#include "common.cuh"
#include "fft.cuh"

namespace fsei {

// ------------------------------------------------------- kernel entries ----
// The kernels of a step are __device__ bodies with two entry points: k_solo
// runs a body for one grid with its arguments as kernel parameters; k_group
// runs it for the boxes of a batch group at once, box blockIdx.z taking its
// arguments from row blockIdx.z of a table that travels as one by-value
// kernel parameter (every box of a group has the same extents, so the same
// launch shape).  Both entries read their arguments from the constant bank,
// so the group entry needs no more registers than the solo one.  A
// Kernel<Body, MAXT, MINB> names a body with the launch bounds of both.
template <auto Body, int MAXT, int MINB, typename... P>
__global__ void __launch_bounds__(MAXT, MINB) k_solo(P... p) { Body(p...); }

// boxes one group launch can take: kernel parameters are limited to 32764
// bytes
template <typename Tup> constexpr int group_capacity() {
    constexpr int c = (int)(32000 / sizeof(Tup));
    static_assert(c >= 1, "argument tuple too large for a group launch");
    return c > 64 ? 64 : c;
}
template <typename Tup, int NB> struct GroupRows {
    Tup row[NB];
};

template <auto Body, int MAXT, int MINB, typename... P>
__global__ void __launch_bounds__(MAXT, MINB)
    k_group(const __grid_constant__ GroupRows<cuda::std::tuple<P...>,
                                              group_capacity<cuda::std::tuple<P...>>()> rows) {
    cuda::std::apply(Body, rows.row[blockIdx.z]);
}

// One launch of a fractional step as recorded for a batch group: the entry
// of its body, launch shape, stream and the bytes of its argument tuple (a
// cuda::std::tuple of the body's parameter types, identical on the host and
// the device); or a memset, or the fork / join of the grid's side stream.
struct RecordedOp {
    enum Kind { KERNEL, MEMSET, FORK, JOIN } kind;
    cudaStream_t st;
    const void *entry;   // solo entry of the body (identifies the kernel)
    // launches the group entry for nbox <= group_cap boxes whose argument
    // rows (args of each box, back to back) start at rows
    void (*launch_group)(const void *rows, int nbox, dim3 grid, dim3 block, size_t smem,
                         cudaStream_t st, bool pdl);
    void (*prepare_group)();   // loads the group entry, raises its smem limit
    int group_cap;
    dim3 grid, block;
    size_t smem;
    bool pdl;
    std::vector<unsigned char> args;
    void *mem;
    size_t mem_bytes;
};
struct LaunchRecorder {
    std::vector<RecordedOp> ops;
};
// While a recorder is set on the calling host thread, Kernel::launch,
// memset_async and the side-stream fork / join record instead of issuing.
LaunchRecorder *&launch_recorder();

// Launch of kernel k on st; with pdl, as a programmatic dependent launch:
// the grid may be scheduled while the stream's previous kernel finishes (the
// kernel's pdl_wait() holds its blocks until that kernel has completed), so
// the launch latency and the block ramp-up overlap the predecessor's last
// wave.  The launch error, if any, is left for cudaGetLastError.
template <typename... KP, typename... A>
inline void launch_k(bool pdl, void (*k)(KP...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t st, A &&...args) {
    if (pdl) {
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...) == cudaSuccess) return;
        cudaGetLastError();   // the ordinary launch below reports the error
    }
    k<<<grid, block, smem, st>>>(std::forward<A>(args)...);
}

// Largest dynamic shared memory a block may opt into on the current device.
inline int smem_optin() {
    int dev = 0, v = 48 * 1024;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

// Raise a kernel's dynamic shared memory limit to what the device allows
// next to the kernel's static shared memory.  Every kernel's
// MaxDynamicSharedMemorySize attribute is raised to it: the attribute is per
// kernel and process-wide, so a value sized for one grid would cap the
// launches of another grid of the same kernel.
template <typename F> inline void raise_smem_limit(F *kernel) {
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, kernel) != cudaSuccess) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem_optin() - (int)a.sharedSizeBytes);
}

template <auto Body, int MAXT, int MINB, typename... P>
void group_launch_of(const void *rows, int nbox, dim3 grid, dim3 block, size_t smem,
                     cudaStream_t st, bool pdl) {
    using Tup = cuda::std::tuple<P...>;
    constexpr int NB = group_capacity<Tup>();
    static thread_local GroupRows<Tup, NB> t;   // 32 KB at most
    if (nbox < 1 || nbox > NB) return;
    memcpy(&t, rows, sizeof(Tup) * (size_t)nbox);
    grid.z = (unsigned)nbox;
    launch_k(pdl, k_group<Body, MAXT, MINB, P...>, grid, block, smem, st, t);
}
template <auto Body, int MAXT, int MINB, typename... P> void group_prepare_of() {
    raise_smem_limit(k_group<Body, MAXT, MINB, P...>);
}

template <auto Body, int MAXT, int MINB, typename... P>
constexpr auto solo_entry_of(void (*)(P...)) {
    return &k_solo<Body, MAXT, MINB, P...>;
}

template <auto Body, int MAXT, int MINB, typename... P, typename... A>
void launch_body(void (*)(P...), bool pdl, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                 A &&...args) {
    if (LaunchRecorder *rec = launch_recorder()) {
        using Tup = cuda::std::tuple<P...>;
        const Tup t(static_cast<P>(args)...);
        RecordedOp op = {};
        op.kind = RecordedOp::KERNEL;
        op.st = st;
        op.entry = (const void *)&k_solo<Body, MAXT, MINB, P...>;
        op.launch_group = &group_launch_of<Body, MAXT, MINB, P...>;
        op.prepare_group = &group_prepare_of<Body, MAXT, MINB, P...>;
        op.group_cap = group_capacity<Tup>();
        op.grid = grid;
        op.block = block;
        op.smem = smem;
        op.pdl = pdl;
        op.args.resize(sizeof(Tup));
        memcpy(op.args.data(), &t, sizeof(Tup));
        rec->ops.push_back(std::move(op));
        return;
    }
    launch_k(pdl, &k_solo<Body, MAXT, MINB, P...>, grid, block, smem, st,
             static_cast<P>(args)...);
}

template <auto Body, int MAXT, int MINB> struct Kernel {
    // launch on st (pdl: as a programmatic dependent launch), or record it
    template <typename... A>
    void launch(bool pdl, dim3 grid, dim3 block, size_t smem, cudaStream_t st, A &&...args) const {
        launch_body<Body, MAXT, MINB>(Body, pdl, grid, block, smem, st, std::forward<A>(args)...);
    }
    // the solo entry (for function attributes)
    auto solo() const { return solo_entry_of<Body, MAXT, MINB>(Body); }
};

// cudaMemsetAsync, or recorded
inline void memset_async(void *p, int v, size_t n, cudaStream_t st) {
    if (LaunchRecorder *rec = launch_recorder()) {
        RecordedOp op = {};
        op.kind = RecordedOp::MEMSET;
        op.st = st;
        op.mem = p;
        op.mem_bytes = n;
        rec->ops.push_back(std::move(op));
        (void)v;
        return;
    }
    cudaMemsetAsync(p, v, n, st);
}

// Body force and state fields of one step (device pointers, caller-owned).
template <typename T> struct Fields {
    T *u, *v, *w, *p, *hu, *hv, *hw;
    const T *fx, *fy, *fz;   // may be NULL
    // an explicit term added to H at the u, v, w points (the non-Newtonian
    // stress remainder), or NULL
    const T *hx, *hy, *hz;
};

// The two z-sweep plans of a grid (centres, faces) and their storage: what
// the per-step factorisation kernel needs of the workspace.
template <typename T> struct ZPlans {
    TriPlan<T> plan[2];
    TriPlanStore<T> store[2];
};

// Library-owned workspace and launch configuration of one grid.
template <typename T> struct Work {
    T *q0, *q1, *q2;         // sweep intermediates, then u* (3 fields)
    T *phi;                  // pressure increment (1 field)
    cplx<T> *spec;           // spectrum [nz][ny][sk]
    TriPlanStore<T> store[4];
    TriPlan<T> plan[4];      // 0: x, 1: y, 2: z at centres, 3: z at faces
    FftPlanDev fpx, fpy;     // x: length nx/2, y: length ny
    const cplx<T> *twx, *twy, *twpost;   // w^m tables; twpost[k] =
                                          // exp(-2 pi i k / nx), k <= nx/2
    const T *lamx, *lamy;    // modified wavenumbers (sk and ny entries)
    const double *lamx_d, *lamy_d;
    const int *nzm;          // near-zero modes to solve in double: kx + sk*ky
    int n_nzm;
    // Factors of the exactly solved modes' z systems (grid constants, set at
    // grid creation; NULL selects the on-the-fly k_poisson_exact): per mode
    // m and rows i < nz, xa[m nz + i] = -a_i / den_i, xm = 1 / den_i,
    // xc = c_i / den_i of Thomas' algorithm (cyclic lines: of the
    // Sherman-Morrison modified matrix, with xz its solution for the
    // correction vector and xs[2 m], xs[2 m + 1] = v_last, 1 / (1 + v.z)).
    const double *xa, *xm, *xc, *xz, *xs;
    double zlen;             // z extent (sum of dz)
    const unsigned char *exact;   // [ny][sk]: 1 for the modes in nzm
    T *adj0, *adj1, *adj2;   // adjoint workspace (allocated on first use)
    T *nn0, *nn1, *nn2, *nuc;   // non-Newtonian remainder at the u, v, w points
                                // and the excess viscosity at the centres
                                // (allocated on first use)
    int ry;                  // rows per block of the x-line solves
    int ry_fft;              // rows per block of the x transforms
    int chunk_y, chunk_z;    // register chunk length of the y / z sweeps
    int tx_y, tx_z;          // x lanes per block of the y / z sweeps
    int zsw_cols;            // x columns per lane of the z sweep (1 or 2;
                             // 0: 1)
    int py;                  // chunks per y line
    int px, chunk_x;         // chunks per x line and their length (x solves)
    int tkx;                 // kx columns per block of the y FFT / z Poisson
    int pz_poisson;          // chunks per z line in the Poisson solve
    int zl_lpl, zl_e;        // lane-resident z solve: lanes per mode line and
                             // rows per lane (0: not used)
    int rhs_cpl;             // cells per lane of the row-resident RHS (2, 4
                             // or 8; 0: by row width)
    int rhs_strip;           // rows per strip of the RHS marched along y
                             // (0: one row per lane, k_rhs_x_row)
    int proj_mult;           // row passes per thread of the projection (0: 4)
    int ry_rfft;             // rows per block of the forward x transform
    int tkx_fft;             // kx columns per block of the two-pass y
                             // transform
    int pdl;                 // launch the step's kernels as programmatic
                             // dependent launches (launch_k)
};

// Launch schedule of a grid: the tile shapes and solver splits that its
// tunable kernels run with.  Every candidate value of a field computes the
// same quantities with the same operations, grouped differently, so results
// agree to rounding and the choice only moves time.  0 marks a field whose
// kernel does not apply to the grid.
struct Schedule {
    int rhs_cpl;    // RHS + x sweep: cells per lane of the row-resident kernel
    int rhs_strip;  // and rows per strip when marched along y (0: not)
    int zsw_cols;   // z sweep: x columns per lane (1 or 2)
    int zl_lpl;     // z Poisson: lanes per mode line (the reduction across
                    // lanes); zl_e: rows per lane (the elimination in a lane)
    int zl_e;
    int ry_rfft;    // forward x transform: grid rows per block
    int tkx_fft;    // y transforms: kx columns per block
    int proj_mult;  // projection: row passes per thread
};
enum ScheduleKnob { SK_RHS, SK_ZL, SK_RFFT, SK_FFTY, SK_PROJ, SK_ZSW, SK_COUNT };
// the values knob k may take on this grid (pairs (lanes, rows) for SK_ZL,
// (cells per lane, rows per strip) for SK_RHS, single values in out[i][0]
// otherwise), the default first; their count
template <typename T> int schedule_candidates(const GridDev &g, int knob, int (*out)[2], int cap);
template <typename T> Schedule schedule_of(const GridDev &g, const Work<T> &W);
template <typename T> void apply_schedule(Work<T> &W, const Schedule &s);

// Parameters of one fractional step or sub-step.  dt and cfl give the time
// step dt_n of the full step (dt, or cfl / speed of u^n, formed at substep
// 0); the fractional step itself advances by alpha dt_n with the
// Adams-Bashforth-style weights gamma, rho: with alpha = 1 and substep = 0
// that is Eq. 3, and the Runge-Kutta sub-steps pass alpha_l and
// gamma_l / alpha_l, rho_l / alpha_l (their advection weights relative to
// the sub-interval).
struct StepArgs {
    double re, dt, cfl, gamma, rho;
    double fconst[3];
    int scheme;      // fsei_scheme
    int rheology;    // fsei_rheology
    double cy[4];    // Carreau-Yasuda lambda, n, a, eta_inf
    double alpha;    // fraction of dt_n this fractional step covers
    int substep;     // 0: forms dt_n; > 0: reuses it
};
// The three sub-steps of the third-order Runge-Kutta scheme: advection
// weights gamma_l (this sub-step) and rho_l (previous one); the linear terms
// over alpha_l = gamma_l + rho_l of the step.
constexpr double kRk3Gamma[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
constexpr double kRk3Rho[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};

template <typename T> void launch_speed(const GridDev &g, const T *u, const T *v, const T *w,
                                        StepScalars *sc, cudaStream_t st);
template <typename T> void launch_step_begin(const GridDev &g, Work<T> &W, StepScalars *sc,
                                             const StepArgs &a, int euler, cudaStream_t st);
// the two halves of launch_step_begin: this step's scalars (dt, beta, AB2
// weights, reset reductions), then the z-sweep plans that depend on beta
// (needed from the z sweep on, so they may run beside the RHS and y sweep)
void launch_step_scalars(const GridDev &g, StepScalars *sc, const StepArgs &a, int euler,
                         cudaStream_t st, bool pdl = false);
template <typename T> void launch_step_plans(const GridDev &g, Work<T> &W, const StepScalars *sc,
                                             cudaStream_t st);

// A second stream of a grid and two events for a fork-join around work that
// may run beside the main chain (its launches stay stream-ordered, also
// inside a graph capture).
struct Overlap {
    cudaStream_t side;
    cudaEvent_t fork, join;
};
// Let o.side start after the work queued on st so far (fork), or let st
// continue after the work queued on o.side (join); recorded when a
// recorder is set.
inline void fork_side(const Overlap &o, cudaStream_t st) {
    if (LaunchRecorder *rec = launch_recorder()) {
        RecordedOp op = {};
        op.kind = RecordedOp::FORK;
        op.st = st;
        rec->ops.push_back(std::move(op));
        return;
    }
    cudaEventRecord(o.fork, st);
    cudaStreamWaitEvent(o.side, o.fork, 0);
}
inline void join_side(const Overlap &o, cudaStream_t st) {
    if (LaunchRecorder *rec = launch_recorder()) {
        RecordedOp op = {};
        op.kind = RecordedOp::JOIN;
        op.st = st;
        rec->ops.push_back(std::move(op));
        return;
    }
    cudaEventRecord(o.join, o.side);
    cudaStreamWaitEvent(st, o.join, 0);
}
template <typename T> void launch_rhs_x(const GridDev &g, const Fields<T> &F, Work<T> &W,
                                        const StepScalars *sc, const StepArgs &a, cudaStream_t st);
// the marched RHS (k_rhs_march.cu) with W.rhs_cpl and W.rhs_strip; false
// (nothing launched) where that layout does not apply
template <typename T>
bool launch_rhs_x_march(const GridDev &g, const Fields<T> &F, Work<T> &W, const StepScalars *sc,
                        const StepArgs &a, cudaStream_t st);
template <typename T> void launch_sweep_y(const GridDev &g, Work<T> &W, const StepScalars *sc,
                                          cudaStream_t st);
template <typename T> void launch_sweep_z(const GridDev &g, const Fields<T> &F, Work<T> &W,
                                          cudaStream_t st);
// mode 0: s = D(q0,q1,q2) / dt ; mode 1: s = the given field src (scaled 1)
template <typename T> void launch_rfft_x(const GridDev &g, Work<T> &W, const StepScalars *sc,
                                         const T *src, int mode, cudaStream_t st);
template <typename T> void launch_fft_y(const GridDev &g, Work<T> &W, int inverse, cudaStream_t st);
// compat = 1: the (0, 0) mode's right-hand side first loses its dz-weighted
// mean (an arbitrary right-hand side made compatible; used by the adjoint)
template <typename T> void launch_poisson_z(const GridDev &g, Work<T> &W, cudaStream_t st,
                                            int compat = 0);
template <typename T> void launch_irfft_x(const GridDev &g, Work<T> &W, T *dst, cudaStream_t st);
// z sweep of the adjoint: q = W (I - beta L_z)^-1 q, W = dz_k (u, v) or
// hc_k (w)
template <typename T> void launch_sweep_z_adjoint(const GridDev &g, Work<T> &W, cudaStream_t st);
// Optional hook around the launch groups of a multi-kernel launcher (used
// for per-kernel timing): before(ctx, kind, st) and after(ctx, kind, st)
// bracket the launches of group `kind` on st.
struct LaunchHook {
    void *ctx;
    void (*before)(void *ctx, int kind, cudaStream_t st);
    void (*after)(void *ctx, int kind, cudaStream_t st);
};
// launch groups of the adjoint step, in call order
enum AdjointKind {
    AK_PHIBAR, AK_POISSON, AK_USTAR, AK_SWEEP_Z, AK_SWEEP_Y, AK_SWEEP_X, AK_HIST, AK_GATHER,
    AK_COUNT
};
template <typename T>
void launch_adjoint_step(const GridDev &g, Work<T> &W, StepScalars *sc, const T *u, const T *v,
                         const T *w, T *ub, T *vb, T *wb, T *pb, T *hbu, T *hbv, T *hbw, T *fbx,
                         T *fby, T *fbz, double re, cudaStream_t st,
                         const LaunchHook *hook = nullptr);
template <typename T> void set_smem_limits_adjoint(const GridDev &g, const Work<T> &W);
// immersed-boundary forcing of nm markers (k_ib.cu): interpolate, force,
// spread into fx, fy, fz (+=); u_at (nullable): interpolated velocities
// (nm x 3); skipped[0] counts markers whose support leaves the interior
template <typename T>
void launch_ib_force(const GridDev &g, const T *u, const T *v, const T *w, const double *xb,
                     const double *ub, const double *dvb, int nm, double dt, T *fx, T *fy,
                     T *fz, double *u_at, int *skipped, cudaStream_t st);
// face loads (face_force written, node_force += a third per node);
// skipped[0] counts faces whose probe support leaves the interior,
// skipped[1] node indices outside [0, nnodes)
template <typename T>
void launch_ib_loads(const GridDev &g, const T *p, const T *u, const T *v, const T *w,
                     const double *xf, const double *nf, const double *af, const int *two_sided,
                     const int *tris, int nfaces, int nnodes, double probe, double inv_re,
                     double *face_force, double *node_force, int *skipped, cudaStream_t st);
template <typename T> void preload_ib();
// the Carreau-Yasuda remainder div(2 Re^-1 (eta - 1) E) of (u, v, w) into
// W.nn0..2 (k_rheology.cu); cy: lambda, n, a, eta_inf
template <typename T>
void launch_non_newtonian(const GridDev &g, const T *u, const T *v, const T *w, Work<T> &W,
                          double re, const double cy[4], cudaStream_t st);
template <typename T> void preload_rheology();
template <typename T> void preload_project();
template <typename T> void launch_project(const GridDev &g, const Fields<T> &F, Work<T> &W,
                                          StepScalars *sc, cudaStream_t st);


// dynamic shared memory bytes of each kernel (host-side sizing helpers)
template <typename T> size_t smem_rhs_x(const GridDev &g, const Work<T> &W);
template <typename T> size_t smem_fft_x(const GridDev &g, const Work<T> &W);
template <typename T> size_t smem_fft_y(const GridDev &g, const Work<T> &W);
template <typename T> size_t smem_poisson(const GridDev &g, const Work<T> &W);
template <typename T> void set_smem_limits_sweep(const GridDev &g, const Work<T> &W);
template <typename T> void set_smem_limits_march(const GridDev &g, const Work<T> &W);
template <typename T> void set_smem_limits_lines(const GridDev &g, const Work<T> &W);
// chunk length, chunks per line and x columns per block of the register
// sweeps for lines of n unknowns
void sweep_geometry(int n, int &chunk, int &P, int &tx);
// the same for the uniform periodic y sweep (uni_solve)
void sweep_y_geometry(int n, int &chunk, int &P, int &tx);
// chunks per line P (a power of two <= 32 with nl P <= maxthr) and chunk
// length for nl uniform periodic lines of n unknowns solved by one block
void uni_geometry(int n, int nl, int maxthr, int &P, int &chunk);
template <typename T> void set_smem_limits_poisson(const GridDev &g, const Work<T> &W);
// rows per block of the x transforms, kx columns per block of the y
// transform and z solve, chunks per z line of the z solve (sets ry_fft, tkx,
// pz_poisson)
template <typename T> void poisson_geometry(const GridDev &g, Work<T> &W);
// the (lanes per line, rows per lane) splits of the lane-resident z solve
// that apply to this grid, in order of preference (at most cap); their count
int zl_candidates(const GridDev &g, int elem_size, int (*out)[2], int cap);
// cells per lane of the row-resident RHS that apply to this grid (at most
// cap); their count
int rhs_cpl_candidates(const GridDev &g, int elem_size, int *out, int cap);
// row layout of the row-resident RHS: cpl cells per lane (prefer, or by
// row width), lpr lanes per row, rpb rows per block; false where it does not
// apply
template <typename T>
bool rhs_row_geometry(const GridDev &g, int &cpl, int &lpr, int &rpb, int prefer = 0);
// whether the marched RHS takes strips of S rows with cpl cells per lane
// (0: by row width) on this grid
bool rhs_strip_admissible(const GridDev &g, int elem_size, int cpl, int S);

}  // namespace fsei
