// Host side of libfsei.so: the C ABI of include/fsei.h.  Builds the mesh
// metrics, FFT twiddle tables, Fourier-mode tables and workspace of a grid,
// and sequences the kernels of a fractional step (Sec. 2.1, Eq. 3; Sec. 3.1).
#include <math.h>
#include <nvtx3/nvToolsExt.h>
#include <stdlib.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/fsei.h"
#include "kernels.cuh"

using namespace fsei;

namespace fsei {
LaunchRecorder *&launch_recorder() {
    static thread_local LaunchRecorder *rec = nullptr;
    return rec;
}
}  // namespace fsei

namespace {

thread_local std::string g_err;

fsei_status fail(fsei_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

bool is_2a3b(int n) {
    if (n < 1) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

FftPlanDev make_fft_plan(int n) {
    FftPlanDev p;
    memset(&p, 0, sizeof p);
    p.n = n;
    int m = n;
    while (m % 4 == 0) { p.rad[p.nr++] = 4; m /= 4; }
    while (m % 2 == 0) { p.rad[p.nr++] = 2; m /= 2; }
    while (m % 3 == 0) { p.rad[p.nr++] = 3; m /= 3; }
    return p;
}

// exp(-2 pi i m / n) in extended precision, rounded to double
void twiddles(int n, int count, std::vector<double> &re, std::vector<double> &im) {
    re.resize(count);
    im.resize(count);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int m = 0; m < count; ++m) {
        const long double ang = 2.0L * pi * (long double)m / (long double)n;
        re[m] = (double)cosl(ang);
        im[m] = (double)(-sinl(ang));
    }
}

// Byte pattern of the guard zones around a buffer of element type X in the
// bounds-checking mode: all-ones bytes (a NaN in float and double, so a read
// of a guard turns the results it feeds non-finite) for floating-point
// buffers; zero bytes for integer and mixed ones, so that an index read from
// a guard is still an index inside the grid.
template <typename X> struct GuardFill { static constexpr unsigned char value = 0x00; };
template <> struct GuardFill<float> { static constexpr unsigned char value = 0xFF; };
template <> struct GuardFill<double> { static constexpr unsigned char value = 0xFF; };
template <> struct GuardFill<cplx<float>> { static constexpr unsigned char value = 0xFF; };
template <> struct GuardFill<cplx<double>> { static constexpr unsigned char value = 0xFF; };

// Device allocations of one grid.  limit caps their sum: an allocation
// that would pass it fails like a cudaMalloc without room (a grid created
// under FSEI_WORKSPACE_LIMIT_BYTES, see fsei_grid_create).
//
// Bounds-checking mode (guard = true; FSEI_CHECK_BOUNDS=1 in the
// environment when the grid is created): every buffer sits between two
// guard zones of G = clamp(bytes / 16, 64 KiB, 1 MiB) bytes, rounded to 256,
// filled with the buffer type's GuardFill pattern.  check_guards() reads
// them back: a kernel that wrote up to G bytes past either end of a buffer
// has changed one.  The returned address stays 256-byte aligned.
struct DevAllocs {
    std::vector<void *> ptrs;
    size_t bytes = 0;
    size_t limit = ~size_t(0);
    cudaError_t err = cudaSuccess;
    bool guard = false;
    struct Zone {
        const unsigned char *front, *back;   // device addresses
        size_t gbytes, bytes;                 // guard size, buffer size
        unsigned char fill;
    };
    std::vector<Zone> zones;
    template <typename X> X *get(size_t count) {
        void *p = nullptr;
        const size_t b = (count ? count : 1) * sizeof(X);
        if (b > limit - bytes) {
            err = cudaErrorMemoryAllocation;
            return nullptr;
        }
        const size_t gb = guard ? std::min<size_t>(std::max<size_t>((b / 16 + 255) & ~size_t(255),
                                                                    size_t(64) << 10),
                                                   size_t(1) << 20)
                                : 0;
        cudaError_t e = cudaMalloc(&p, b + 2 * gb);
        if (e != cudaSuccess) {
            err = e;
            return nullptr;
        }
        ptrs.push_back(p);
        bytes += b;
        if (!guard) return static_cast<X *>(p);
        unsigned char *base = static_cast<unsigned char *>(p);
        const unsigned char fill = GuardFill<X>::value;
        e = cudaMemset(base, fill, gb);
        if (e == cudaSuccess) e = cudaMemset(base + gb + b, fill, gb);
        if (e != cudaSuccess) {
            err = e;
            return nullptr;
        }
        zones.push_back({base, base + gb + b, gb, b, fill});
        return reinterpret_cast<X *>(base + gb);
    }
    // First changed guard byte: buffer index (allocation order), side
    // (0 before, 1 after the buffer) and byte offset from the buffer's
    // edge; false when every guard is intact.  Synchronises the device.
    bool check_guards(size_t *buf, int *side, size_t *offset, cudaError_t *cerr) const {
        *cerr = cudaDeviceSynchronize();
        if (*cerr != cudaSuccess) return false;
        std::vector<unsigned char> h;
        for (size_t i = 0; i < zones.size(); ++i) {
            const Zone &z = zones[i];
            h.resize(z.gbytes);
            for (int sd = 0; sd < 2; ++sd) {
                *cerr = cudaMemcpy(h.data(), sd ? z.back : z.front, z.gbytes,
                                   cudaMemcpyDeviceToHost);
                if (*cerr != cudaSuccess) return false;
                // nearest the buffer first: the back guard from its start,
                // the front guard from its end
                for (size_t d = 0; d < z.gbytes; ++d) {
                    if (h[sd ? d : z.gbytes - 1 - d] != z.fill) {
                        *buf = i;
                        *side = sd;
                        *offset = d;
                        return true;
                    }
                }
            }
        }
        return false;
    }
    void release() {
        for (void *p : ptrs) cudaFree(p);
        ptrs.clear();
        zones.clear();
    }
};

enum KernelKind {
    KK_SPEED, KK_BEGIN, KK_RHS_X, KK_SWEEP_Y, KK_SWEEP_Z, KK_RFFT_X, KK_FFT_Y, KK_POISSON_Z,
    KK_IFFT_Y, KK_IRFFT_X, KK_PROJECT, KK_PLANS, KK_NN,
    // the adjoint step's launch groups (AdjointKind order)
    KK_ADJ_FIRST, KK_COUNT = KK_ADJ_FIRST + AK_COUNT
};
const char *const kKernelNames[KK_COUNT] = {
    "speed (CFL reduction)", "step_begin (scalars)", "rhs_x (RHS + x sweep)",
    "sweep_y", "sweep_z (+ u*)", "rfft_x (div + x R2C)", "fft_y (forward)",
    "poisson_z (+ exact modes)", "fft_y (inverse)", "irfft_x (x C2R)",
    "project (+ p update, stats)", "z-sweep plans (side stream)",
    "non-Newtonian remainder (2 launches)",
    "adj_phibar", "adj_poisson (5 launches)", "adj_ustar", "adj_sweep_z", "adj_sweep_y",
    "adj_sweep_x", "adj_hist", "adj_gather"};

// NVTX ranges: one per public call and one per pass of the step (named as
// the kernel table above names it), so a profiler's timeline shows which
// pass a kernel belongs to.  Host-side annotations only; without an attached
// tool each push or pop is a check of a null function pointer.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Event pairs recorded around kernel launches while timing is enabled.
struct KernelTimer {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<int> kinds;   // kind of pending pair i (events 2i, 2i+1)
    double ms[KK_COUNT] = {0};
    long long n[KK_COUNT] = {0};
    cudaEvent_t ev(size_t i) {
        while (pool.size() <= i) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[i];
    }
    // while capturing a graph: the first launch group that raised an error
    bool check = false;
    int fail_kind = -1;
    cudaError_t fail_err = cudaSuccess;
    template <class F> void run(int kind, cudaStream_t st, F &&f) {
        if (on && !check) {
            begin(kind, st);   // the pass's NVTX range and event pair
            f();
            end(st);
            return;
        }
        NvtxRange range(kKernelNames[kind]);
        if (check) {
            f();
            const cudaError_t e = cudaPeekAtLastError();
            if (e != cudaSuccess && fail_kind < 0) {
                fail_kind = kind;
                fail_err = e;
            }
            return;
        }
        f();
    }
    // the two halves of run(), for launchers in other files (LaunchHook)
    void begin(int kind, cudaStream_t st) {
        nvtxRangePushA(kKernelNames[kind]);
        if (!on) return;
        const size_t i = kinds.size();
        cudaEventRecord(ev(2 * i), st);
        kinds.push_back(kind);
    }
    void end(cudaStream_t st) {
        nvtxRangePop();
        if (!on || kinds.empty()) return;
        cudaEventRecord(ev(2 * kinds.size() - 1), st);
    }
    void collect() {
        cudaDeviceSynchronize();
        for (size_t i = 0; i < kinds.size(); ++i) {
            float t = 0.f;
            cudaEventElapsedTime(&t, pool[2 * i], pool[2 * i + 1]);
            ms[kinds[i]] += t;
            n[kinds[i]] += 1;
        }
        kinds.clear();
    }
    ~KernelTimer() {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
};

template <typename X> cudaError_t upload(X *dst, const std::vector<X> &src) {
    return cudaMemcpy(dst, src.data(), src.size() * sizeof(X), cudaMemcpyHostToDevice);
}

}  // namespace

struct fsei_grid_s {
    fsei_grid_desc desc;
    int device = 0;
    int prec = 0;
    GridDev g;
    DevAllocs mem;
    Work<float> wf;
    Work<double> wd;
    StepScalars *sc = nullptr;      // device
    StepScalars *sc_host = nullptr; // pinned
    int *ib_count = nullptr;        // device: skipped markers / faces, bad node indices
    KernelTimer timer;
    // side stream and fork/join events: the z-sweep plans run beside the
    // RHS and y sweep
    Overlap ov_plans{};
    // fsei_step_host: copy streams and events, created at its first call
    struct HostLink {
        cudaStream_t h2d = nullptr, d2h = nullptr;
        cudaEvent_t back[7] = {};   // field f's copy to the host has landed
        bool back_valid = false;    // a previous call recorded back[]
        cudaEvent_t entry = nullptr, in = nullptr, rhs = nullptr, step = nullptr, out = nullptr;
        bool out_valid = false;     // out was recorded by a call
    } host;
};

namespace {

fsei_status create_overlap(fsei_grid_s *G) {
    cudaStream_t side = nullptr;
    if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess)
        return fail(FSEI_E_CUDA, "side stream creation failed");
    G->ov_plans.side = side;
    cudaEvent_t *evs[2] = {&G->ov_plans.fork, &G->ov_plans.join};
    for (cudaEvent_t *e : evs)
        if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess)
            return fail(FSEI_E_CUDA, "event creation failed");
    return FSEI_OK;
}

fsei_status create_host_link(fsei_grid_s *G) {
    auto &H = G->host;
    if (H.h2d) return FSEI_OK;
    if (cudaStreamCreateWithFlags(&H.h2d, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&H.d2h, cudaStreamNonBlocking) != cudaSuccess)
        return fail(FSEI_E_CUDA, "copy stream creation failed");
    cudaEvent_t *evs[12] = {&H.entry, &H.in, &H.rhs, &H.step, &H.out};
    for (int f = 0; f < 7; ++f) evs[5 + f] = &H.back[f];
    for (cudaEvent_t *e : evs)
        if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess)
            return fail(FSEI_E_CUDA, "event creation failed");
    return FSEI_OK;
}

void destroy_host_link(fsei_grid_s *G) {
    auto &H = G->host;
    cudaEvent_t evs[12] = {H.entry, H.in, H.rhs, H.step, H.out};
    for (int f = 0; f < 7; ++f) evs[5 + f] = H.back[f];
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    if (H.h2d) cudaStreamDestroy(H.h2d);
    if (H.d2h) cudaStreamDestroy(H.d2h);
    H = fsei_grid_s::HostLink{};
}

void destroy_overlap(fsei_grid_s *G) {
    cudaEvent_t evs[2] = {G->ov_plans.fork, G->ov_plans.join};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    if (G->ov_plans.side) cudaStreamDestroy(G->ov_plans.side);
    G->ov_plans = Overlap{};
}

}  // namespace

namespace {

// Thomas factors of the z systems of the exactly solved Poisson modes
// (grid constants), in extended precision: per mode the rows i < n of
// (L_z - lambda) phi = s (the (0, 0) mode: rows k = 1 .. nz-1 with phi_0 = 0)
// and, for cyclic lines, the Sherman-Morrison data; layout as Work::xa.
struct ExactFactors {
    std::vector<double> xa, xm, xc, xz, xs;
};

ExactFactors exact_factors(int nz, bool walls, const std::vector<double> &idz,
                           const std::vector<double> &ihc, const std::vector<double> &lamx,
                           const std::vector<double> &lamy, int sk, const std::vector<int> &nzm) {
    typedef long double R;
    ExactFactors f;
    const size_t nm = nzm.size();
    f.xa.assign(nm * nz, 0.0);
    f.xm.assign(nm * nz, 0.0);
    f.xc.assign(nm * nz, 0.0);
    f.xz.assign(nm * nz, 0.0);
    f.xs.assign(2 * nm, 0.0);
    auto acut = [&](int k) -> R { return (walls && k == 0) ? 0.0L : (R)ihc[k] * (R)idz[k]; };
    auto ccut = [&](int k) -> R {
        return (walls && k == nz - 1) ? 0.0L : (R)ihc[k + 1] * (R)idz[k];
    };
    for (size_t m = 0; m < nm; ++m) {
        const int kx = nzm[m] % sk, ky = nzm[m] / sk;
        const bool zero = kx == 0 && ky == 0;
        const bool cyclic = !walls && !zero;
        const int shift = zero ? 1 : 0, n = nz - shift;
        const R lam = (R)lamx[kx] + (R)lamy[ky];
        std::vector<R> a(n), b(n), c(n), xa(n), xm(n), xc(n);
        for (int i = 0; i < n; ++i) {
            const int k = i + shift;
            a[i] = acut(k);
            c[i] = ccut(k);
            b[i] = -(acut(k) + ccut(k)) - lam;
        }
        R gam = 0.0L;
        if (cyclic) {
            gam = -b[0];
            b[0] -= gam;
            b[n - 1] -= a[0] * c[n - 1] / gam;
        }
        for (int i = 0; i < n; ++i) {
            const R den = i == 0 ? b[0] : b[i] - a[i] * xc[i - 1];
            xm[i] = 1.0L / den;
            xa[i] = i == 0 ? 0.0L : -a[i] * xm[i];
            xc[i] = i == n - 1 ? 0.0L : c[i] * xm[i];
        }
        const size_t o = m * (size_t)nz;
        for (int i = 0; i < n; ++i) {
            f.xa[o + i] = (double)xa[i];
            f.xm[o + i] = (double)xm[i];
            f.xc[o + i] = (double)xc[i];
        }
        if (cyclic) {
            // z = T^-1 u, u = (gamma, 0, ..., 0, c_{n-1})
            std::vector<R> z(n);
            for (int i = 0; i < n; ++i) {
                const R ui = i == 0 ? gam : (i == n - 1 ? c[n - 1] : 0.0L);
                z[i] = (i == 0 ? 0.0L : xa[i] * z[i - 1]) + xm[i] * ui;
            }
            for (int i = n - 2; i >= 0; --i) z[i] -= xc[i] * z[i + 1];
            const R vl = a[0] / gam;
            for (int i = 0; i < n; ++i) f.xz[o + i] = (double)z[i];
            f.xs[2 * m] = (double)vl;
            f.xs[2 * m + 1] = (double)(1.0L / (1.0L + z[0] + vl * z[n - 1]));
        }
    }
    return f;
}

template <typename T>
fsei_status setup_work(fsei_grid_s *G, Work<T> &W, const std::vector<double> &lamx,
                       const std::vector<double> &lamy, const std::vector<int> &nzm,
                       const std::vector<double> &dz, const std::vector<double> &idz,
                       const std::vector<double> &ihc) {
    GridDev &g = G->g;
    DevAllocs &M = G->mem;
    const size_t ncell = (size_t)g.nx * g.ny * g.nz;
    memset(&W, 0, sizeof W);
    W.q0 = M.get<T>(ncell);
    W.q1 = M.get<T>(ncell);
    W.q2 = M.get<T>(ncell);
    W.phi = M.get<T>(ncell);
    const size_t nspec = (size_t)g.sk * g.ny * g.nz;
    W.spec = M.get<cplx<T>>(nspec);
    if (M.err != cudaSuccess) return fail(FSEI_E_NOMEM, "workspace allocation failed (%zu bytes so far): %s", M.bytes, cudaGetErrorString(M.err));
    cudaMemset(W.spec, 0, nspec * sizeof(cplx<T>));

    // launch geometry
    const int tsz = (int)sizeof(T);
    W.ry = 1;
    for (int r = 4; r >= 1; r /= 2)
        if (g.ny % r == 0) { W.ry = r; break; }
    poisson_geometry<T>(g, W);
    // x lines (uniform, periodic): 3 ry lines of a block, chunks of at most
    // 64 unknowns (fewer rows per block for the widest meshes)
    uni_geometry(g.nx, 3 * W.ry, 256, W.px, W.chunk_x);
    while (W.chunk_x > 64 && W.ry > 1) {
        W.ry /= 2;
        uni_geometry(g.nx, 3 * W.ry, 256, W.px, W.chunk_x);
    }
    sweep_y_geometry(g.ny, W.chunk_y, W.py, W.tx_y);
    // tridiagonal plans of the z lines: 2 centres, 3 faces (entries 0 and 1
    // are unused: the x and y lines need no plan)
    int Ps[4] = {1, 1, 1, 1};
    // the wall-bounded face lines (w, faces 1 .. nz-1) get one padding
    // unknown: nz like the centre lines, so both split into equal chunks
    int ns[4] = {g.nx, g.ny, g.nz, g.nz};
    {
        int cz, pz, tz, cf, pf, tf;
        sweep_geometry(ns[2], cz, pz, tz);
        sweep_geometry(ns[3], cf, pf, tf);
        Ps[2] = pz;
        Ps[3] = pf;
        W.chunk_z = cz > cf ? cz : cf;
        W.tx_z = tz < tf ? tz : tf;
    }
    for (int q = 2; q < 4; ++q) {
        if (Ps[q] > ns[q] / 3) Ps[q] = ns[q] / 3;
        if (Ps[q] < 1) Ps[q] = 1;
        TriPlanStore<T> &s = W.store[q];
        const int n = ns[q], m = 2 * Ps[q];
        s.a = M.get<T>(n); s.c = M.get<T>(n); s.inv = M.get<T>(n);
        s.at = M.get<T>(n); s.ct = M.get<T>(n);
        s.rlo = M.get<T>(m); s.rinv = M.get<T>(m); s.rcp = M.get<T>(m);
        s.rz = M.get<T>(m); s.rsc = M.get<T>(2);
        s.pk1 = M.get<T>(kPcrLevels * m); s.pk2 = M.get<T>(kPcrLevels * m);
        s.pdinv = M.get<T>(m);
        TriPlan<T> &p = W.plan[q];
        p.n = n;
        p.P = Ps[q];
        p.cyclic = (q < 2) ? 1 : (g.walls ? 0 : 1);
        p.off = (q == 3 && g.walls) ? 1 : 0;
        p.pad = (q == 3 && g.walls) ? 1 : 0;
        p.a = s.a; p.c = s.c; p.inv = s.inv; p.at = s.at; p.ct = s.ct;
        p.rlo = s.rlo; p.rinv = s.rinv; p.rcp = s.rcp; p.rz = s.rz; p.rsc = s.rsc;
        p.pk1 = s.pk1; p.pk2 = s.pk2; p.pdinv = s.pdinv;
        p.levels = 0;
        if (m <= 128 && (m & (m - 1)) == 0)
            while ((1 << p.levels) < m) ++p.levels;
    }
    if (M.err != cudaSuccess) return fail(FSEI_E_NOMEM, "plan allocation failed");

    // FFT plans and twiddles
    W.fpx = make_fft_plan(g.mx);
    W.fpy = make_fft_plan(g.ny);
    auto up_tw = [&](int n, int count, const cplx<T> **dst) {
        std::vector<double> re, im;
        twiddles(n, count, re, im);
        std::vector<cplx<T>> h(count);
        for (int m = 0; m < count; ++m) h[m] = cplx<T>{T(re[m]), T(im[m])};
        cplx<T> *d = M.get<cplx<T>>(count);
        if (d) upload(d, h);
        *dst = d;
    };
    up_tw(g.mx, g.mx, &W.twx);
    up_tw(g.ny, g.ny, &W.twy);
    up_tw(g.nx, g.mx + 1, &W.twpost);
    // modified wavenumbers
    {
        std::vector<T> lx(lamx.size()), ly(lamy.size());
        for (size_t i = 0; i < lamx.size(); ++i) lx[i] = T(lamx[i]);
        for (size_t i = 0; i < lamy.size(); ++i) ly[i] = T(lamy[i]);
        T *dlx = M.get<T>(lx.size());
        T *dly = M.get<T>(ly.size());
        double *dlxd = M.get<double>(lamx.size());
        double *dlyd = M.get<double>(lamy.size());
        int *dm = M.get<int>(nzm.size());
        if (M.err != cudaSuccess) return fail(FSEI_E_NOMEM, "table allocation failed");
        upload(dlx, lx);
        upload(dly, ly);
        upload(dlxd, lamx);
        upload(dlyd, lamy);
        upload(dm, nzm);
        std::vector<unsigned char> flag((size_t)g.sk * g.ny, 0);
        for (int code : nzm) flag[code] = 1;
        unsigned char *dflag = M.get<unsigned char>(flag.size());
        if (M.err != cudaSuccess) return fail(FSEI_E_NOMEM, "table allocation failed");
        upload(dflag, flag);
        W.exact = dflag;
        W.lamx = dlx; W.lamy = dly; W.lamx_d = dlxd; W.lamy_d = dlyd;
        W.nzm = dm;
        W.n_nzm = (int)nzm.size();
    }
    {
        const ExactFactors ef = exact_factors(g.nz, g.walls != 0, idz, ihc, lamx, lamy, g.sk, nzm);
        double *xa = M.get<double>(ef.xa.size()), *xm = M.get<double>(ef.xm.size());
        double *xc = M.get<double>(ef.xc.size()), *xz = M.get<double>(ef.xz.size());
        double *xs = M.get<double>(ef.xs.size());
        if (M.err != cudaSuccess) return fail(FSEI_E_NOMEM, "table allocation failed");
        upload(xa, ef.xa);
        upload(xm, ef.xm);
        upload(xc, ef.xc);
        upload(xz, ef.xz);
        upload(xs, ef.xs);
        W.xa = xa; W.xm = xm; W.xc = xc; W.xz = xz; W.xs = xs;
        double zl = 0.0;
        for (double d : dz) zl += d;
        W.zlen = zl;
    }
    if (M.err != cudaSuccess) return fail(FSEI_E_NOMEM, "table allocation failed");
    set_smem_limits_sweep<T>(g, W);
    set_smem_limits_march<T>(g, W);
    set_smem_limits_lines<T>(g, W);
    set_smem_limits_poisson<T>(g, W);
    set_smem_limits_adjoint<T>(g, W);
    preload_project<T>();
    preload_ib<T>();
    preload_rheology<T>();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FSEI_E_CUDA, "grid setup: %s", cudaGetErrorString(e));
    return FSEI_OK;
}

// the rheology fields of a caller's parameters
fsei_status check_rheology(const fsei_step_params &p, const char *who) {
    if (p.rheology == FSEI_NEWTONIAN) return FSEI_OK;
    if (p.rheology != FSEI_CARREAU_YASUDA) return fail(FSEI_E_ARG, "%s: unknown rheology %d", who, p.rheology);
    if (p.scheme != FSEI_AB2_CN)
        return fail(FSEI_E_UNSUPPORTED, "%s: the Carreau-Yasuda law runs with the Adams-Bashforth scheme only", who);
    if (!(p.cy.lambda >= 0) || !(p.cy.n > 0) || !(p.cy.a > 0) || !(p.cy.eta_inf >= 0) ||
        !(p.cy.eta_inf <= 1))
        return fail(FSEI_E_ARG, "%s: Carreau-Yasuda needs lambda >= 0, n > 0, a > 0, 0 <= eta_inf <= 1", who);
    return FSEI_OK;
}

// StepArgs of a caller's parameters (one Adams-Bashforth step; run_steps
// splits Runge-Kutta steps into their sub-steps)
StepArgs step_args(const fsei_step_params &p) {
    StepArgs a;
    a.re = p.re; a.dt = p.dt; a.cfl = p.cfl; a.gamma = p.gamma; a.rho = p.rho;
    for (int i = 0; i < 3; ++i) a.fconst[i] = p.fconst[i];
    a.scheme = p.scheme;
    a.rheology = p.rheology;
    a.cy[0] = p.cy.lambda; a.cy[1] = p.cy.n; a.cy[2] = p.cy.a; a.cy[3] = p.cy.eta_inf;
    a.alpha = 1.0;
    a.substep = 0;
    return a;
}

template <typename T>
fsei_status run_steps(fsei_grid_s *G, Work<T> &W, fsei_state *s, const void *fx, const void *fy,
                      const void *fz, const StepArgs &a, int nsteps, cudaStream_t st,
                      bool with_speed = true, cudaEvent_t after_rhs = nullptr) {
    Fields<T> F;
    F.u = (T *)s->u; F.v = (T *)s->v; F.w = (T *)s->w; F.p = (T *)s->p;
    F.hu = (T *)s->hu; F.hv = (T *)s->hv; F.hw = (T *)s->hw;
    F.fx = (const T *)fx; F.fy = (const T *)fy; F.fz = (const T *)fz;
    F.hx = F.hy = F.hz = nullptr;
    if (a.rheology == FSEI_CARREAU_YASUDA) {
        if (!W.nn0) {
            const size_t ncell = (size_t)G->g.nx * G->g.ny * G->g.nz;
            W.nn0 = G->mem.get<T>(ncell);
            W.nn1 = G->mem.get<T>(ncell);
            W.nn2 = G->mem.get<T>(ncell);
            W.nuc = G->mem.get<T>(ncell);
            if (G->mem.err != cudaSuccess) {
                W.nn0 = W.nn1 = W.nn2 = W.nuc = nullptr;
                G->mem.err = cudaSuccess;
                return fail(FSEI_E_NOMEM, "non-Newtonian workspace allocation failed");
            }
        }
        F.hx = W.nn0; F.hy = W.nn1; F.hz = W.nn2;
    }
    const GridDev &g = G->g;
    KernelTimer &tm = G->timer;
    // programmatic dependent launches between the step's kernels (in a
    // captured graph they become programmatic edges), except while event
    // pairs time each kernel
    W.pdl = !tm.on ? 1 : 0;
    if (a.cfl > 0.0 && with_speed) {
        memset_async(&G->sc->speed_next, 0, sizeof(unsigned long long), st);
        tm.run(KK_SPEED, st, [&] { launch_speed<T>(g, F.u, F.v, F.w, G->sc, st); });
    }
    const bool rk3 = a.scheme == FSEI_RK3_CN;
    const int subs = rk3 ? 3 : 1;
    for (int n = 0; n < nsteps * subs; ++n) {
        // Eq. 3 (one fractional step), or Runge-Kutta sub-step l = n % 3 as
        // a fractional step over alpha_l dt with weights gamma_l / alpha_l,
        // rho_l / alpha_l (rho_1 = 0: no history needed)
        StepArgs b = a;
        int euler = (n == 0 && !s->have_prev_h) ? 1 : 0;
        if (rk3) {
            const int l = n % 3;
            b.alpha = kRk3Gamma[l] + kRk3Rho[l];
            b.gamma = kRk3Gamma[l] / b.alpha;
            b.rho = kRk3Rho[l] / b.alpha;
            b.substep = l;
            euler = 0;
        }
        tm.run(KK_BEGIN, st, [&] { launch_step_scalars(g, G->sc, b, euler, st, W.pdl != 0); });
        // the z-sweep plans depend on this step's beta and are first read by
        // the z sweep: they run on the side stream beside rhs_x and sweep_y
        const Overlap &op = G->ov_plans;
        fork_side(op, st);
        tm.run(KK_PLANS, op.side, [&] { launch_step_plans<T>(g, W, G->sc, op.side); });
        if (F.hx)
            tm.run(KK_NN, st, [&] {
                launch_non_newtonian<T>(g, F.u, F.v, F.w, W, a.re, a.cy, st);
            });
        tm.run(KK_RHS_X, st, [&] { launch_rhs_x<T>(g, F, W, G->sc, b, st); });
        // H^n is final once the last (sub)step's RHS has run
        if (after_rhs && n == nsteps * subs - 1) cudaEventRecord(after_rhs, st);
        tm.run(KK_SWEEP_Y, st, [&] { launch_sweep_y<T>(g, W, G->sc, st); });
        join_side(op, st);
        tm.run(KK_SWEEP_Z, st, [&] { launch_sweep_z<T>(g, F, W, st); });
        tm.run(KK_RFFT_X, st, [&] { launch_rfft_x<T>(g, W, G->sc, nullptr, 0, st); });
        tm.run(KK_FFT_Y, st, [&] { launch_fft_y<T>(g, W, 0, st); });
        tm.run(KK_POISSON_Z, st, [&] { launch_poisson_z<T>(g, W, st); });
        tm.run(KK_IFFT_Y, st, [&] { launch_fft_y<T>(g, W, 1, st); });
        tm.run(KK_IRFFT_X, st, [&] { launch_irfft_x<T>(g, W, W.phi, st); });
        tm.run(KK_PROJECT, st, [&] { launch_project<T>(g, F, W, G->sc, st); });
    }
    W.pdl = 0;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FSEI_E_CUDA, "step launch: %s", cudaGetErrorString(e));
    return FSEI_OK;
}

template <typename T>
fsei_status run_poisson(fsei_grid_s *G, Work<T> &W, const void *rhs, void *phi, cudaStream_t st) {
    const GridDev &g = G->g;
    KernelTimer &tm = G->timer;
    tm.run(KK_RFFT_X, st, [&] { launch_rfft_x<T>(g, W, G->sc, (const T *)rhs, 1, st); });
    tm.run(KK_FFT_Y, st, [&] { launch_fft_y<T>(g, W, 0, st); });
    tm.run(KK_POISSON_Z, st, [&] { launch_poisson_z<T>(g, W, st); });
    tm.run(KK_IFFT_Y, st, [&] { launch_fft_y<T>(g, W, 1, st); });
    tm.run(KK_IRFFT_X, st, [&] { launch_irfft_x<T>(g, W, (T *)phi, st); });
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FSEI_E_CUDA, "poisson launch: %s", cudaGetErrorString(e));
    return FSEI_OK;
}

// Launch-schedule autotuner.  The schedules measured in this process, by
// grid shape: every grid created later with a tuned shape starts from its
// schedule, so grids of one shape (a batch's boxes, solo runs beside it)
// run the same kernels and give identical results.
using ScheduleKey = std::tuple<int, int, int, int, int, int>;
std::mutex g_sched_mu;
std::map<ScheduleKey, Schedule> g_sched;

ScheduleKey schedule_key(const fsei_grid_s *G) {
    return ScheduleKey(G->device, G->prec, G->g.nx, G->g.ny, G->g.nz, G->g.walls);
}

bool cached_schedule(const fsei_grid_s *G, Schedule *out) {
    std::lock_guard<std::mutex> lk(g_sched_mu);
    auto it = g_sched.find(schedule_key(G));
    if (it == g_sched.end()) return false;
    *out = it->second;
    return true;
}

void store_schedule(const fsei_grid_s *G, const Schedule &s) {
    std::lock_guard<std::mutex> lk(g_sched_mu);
    g_sched[schedule_key(G)] = s;
}

// the kernel kinds whose device time decides knob k
double knob_ms(const KernelTimer &tm, int knob) {
    switch (knob) {
    case SK_RHS: return tm.ms[KK_RHS_X];
    case SK_ZL: return tm.ms[KK_POISSON_Z];
    case SK_RFFT: return tm.ms[KK_RFFT_X];
    case SK_FFTY: return tm.ms[KK_FFT_Y] + tm.ms[KK_IFFT_Y];
    case SK_PROJ: return tm.ms[KK_PROJECT];
    case SK_ZSW: return tm.ms[KK_SWEEP_Z];
    default: return 0.0;
    }
}

void set_knob(Schedule &s, int knob, const int v[2]) {
    switch (knob) {
    case SK_RHS: s.rhs_cpl = v[0]; s.rhs_strip = v[1]; break;
    case SK_ZL: s.zl_lpl = v[0]; s.zl_e = v[1]; break;
    case SK_RFFT: s.ry_rfft = v[0]; break;
    case SK_FFTY: s.tkx_fft = v[0]; break;
    case SK_PROJ: s.proj_mult = v[0]; break;
    case SK_ZSW: s.zsw_cols = v[0]; break;
    default: break;
    }
}

// Times every candidate of every knob in turn (the others held at their
// current choice) inside whole steps on stand-in fields, with the grid's
// kernel timer, and keeps for each knob the candidate of least summed
// device time over `reps` steps (a challenger must beat the incumbent by
// 1%).  The grid's step scalars and timer sums are put back afterwards.
template <typename T>
fsei_status tune_grid(fsei_grid_s *G, Work<T> &W, int reps, cudaStream_t st) {
    const GridDev &g = G->g;
    const size_t ncell = (size_t)g.nx * g.ny * g.nz;
    T *buf = nullptr;
    if (cudaMalloc(&buf, 7 * ncell * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fail(FSEI_E_NOMEM, "autotune: no room for the stand-in fields (%zu bytes)",
                    7 * ncell * sizeof(T));
    }
    // constant fill (0x3c bytes: about 0.0115 in float, 1.6e-18 in double):
    // finite values, the same memory traffic as any other
    cudaMemsetAsync(buf, 0x3c, 7 * ncell * sizeof(T), st);
    fsei_state s;
    s.u = buf; s.v = buf + ncell; s.w = buf + 2 * ncell; s.p = buf + 3 * ncell;
    s.hu = buf + 4 * ncell; s.hv = buf + 5 * ncell; s.hw = buf + 6 * ncell;
    s.have_prev_h = 1;
    fsei_step_params tp = {};
    tp.re = 1000.0; tp.dt = 1e-4; tp.gamma = 1.5; tp.rho = -0.5;
    StepArgs a = step_args(tp);
    a.fconst[0] = a.fconst[1] = a.fconst[2] = 0.0;

    KernelTimer &tm = G->timer;
    tm.collect();
    double ms_keep[KK_COUNT];
    long long n_keep[KK_COUNT];
    memcpy(ms_keep, tm.ms, sizeof ms_keep);
    memcpy(n_keep, tm.n, sizeof n_keep);
    const bool on_keep = tm.on;
    StepScalars sc_keep;
    cudaStreamSynchronize(st);
    cudaMemcpy(&sc_keep, G->sc, sizeof sc_keep, cudaMemcpyDeviceToHost);

    fsei_status r = FSEI_OK;
    Schedule cur = schedule_of<T>(g, W);
    tm.on = true;
    for (int knob = 0; knob < SK_COUNT && r == FSEI_OK; ++knob) {
        int cand[16][2];
        const int nc = schedule_candidates<T>(g, knob, cand, 16);
        if (nc < 2) continue;
        int best = -1;
        double best_ms = 0.0;
        for (int c = 0; c < nc && r == FSEI_OK; ++c) {
            Schedule trial = cur;
            set_knob(trial, knob, cand[c]);
            apply_schedule<T>(W, trial);
            r = run_steps<T>(G, W, &s, nullptr, nullptr, nullptr, a, 1, st, false);
            tm.collect();
            memset(tm.ms, 0, sizeof tm.ms);
            if (r == FSEI_OK) r = run_steps<T>(G, W, &s, nullptr, nullptr, nullptr, a, reps, st, false);
            tm.collect();
            const double t = knob_ms(tm, knob);
            if (best < 0 || t < 0.99 * best_ms) {
                best = c;
                best_ms = t;
            }
        }
        if (best >= 0) set_knob(cur, knob, cand[best]);
    }
    apply_schedule<T>(W, cur);
    tm.on = on_keep;
    memcpy(tm.ms, ms_keep, sizeof ms_keep);
    memcpy(tm.n, n_keep, sizeof n_keep);
    cudaMemcpy(G->sc, &sc_keep, sizeof sc_keep, cudaMemcpyHostToDevice);
    cudaFree(buf);
    const cudaError_t e = cudaGetLastError();
    if (r == FSEI_OK && e != cudaSuccess) r = fail(FSEI_E_CUDA, "autotune: %s", cudaGetErrorString(e));
    if (r == FSEI_OK) store_schedule(G, cur);
    return r;
}

void to_public(const Schedule &s, fsei_schedule *o) {
    o->rhs_cells_per_lane = s.rhs_cpl;
    o->rhs_rows_per_strip = s.rhs_strip;
    o->zsweep_columns_per_lane = s.zsw_cols;
    o->poisson_lanes_per_line = s.zl_lpl;
    o->poisson_rows_per_lane = s.zl_e;
    o->rfft_rows_per_block = s.ry_rfft;
    o->ffty_columns_per_block = s.tkx_fft;
    o->project_passes_per_thread = s.proj_mult;
}

Schedule grid_schedule(const fsei_grid_s *G) {
    return G->prec == FSEI_FP64 ? schedule_of<double>(G->g, G->wd) : schedule_of<float>(G->g, G->wf);
}

void grid_apply(fsei_grid_s *G, const Schedule &s) {
    if (G->prec == FSEI_FP64) apply_schedule<double>(G->wd, s);
    else apply_schedule<float>(G->wf, s);
}

// s holds, for every knob, one of the grid's candidates (0 where the knob has
// none)
bool schedule_valid(const fsei_grid_s *G, const Schedule &s) {
    for (int knob = 0; knob < SK_COUNT; ++knob) {
        int cand[16][2];
        const int nc = G->prec == FSEI_FP64 ? schedule_candidates<double>(G->g, knob, cand, 16)
                                            : schedule_candidates<float>(G->g, knob, cand, 16);
        int v0 = 0, v1 = 0;
        switch (knob) {
        case SK_RHS: v0 = s.rhs_cpl; v1 = s.rhs_strip; break;
        case SK_ZL: v0 = s.zl_lpl; v1 = s.zl_e; break;
        case SK_RFFT: v0 = s.ry_rfft; break;
        case SK_FFTY: v0 = s.tkx_fft; break;
        case SK_PROJ: v0 = s.proj_mult; break;
        case SK_ZSW: v0 = s.zsw_cols; break;
        default: break;
        }
        bool ok = nc == 0 && v0 == 0 && v1 == 0;
        for (int c = 0; c < nc && !ok; ++c)
            ok = cand[c][0] == v0 && cand[c][1] == v1;
        if (!ok) return false;
    }
    return true;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" {

const char *fsei_last_error(void) { return g_err.c_str(); }

const char *fsei_version(void) { return "fsei-gb300 0.1 (sm_103a)"; }

fsei_status fsei_grid_create(const fsei_grid_desc *d, fsei_grid *out) {
    NvtxRange nvtx_call("fsei_grid_create");
    g_err.clear();
    if (!d || !out) return fail(FSEI_E_ARG, "fsei_grid_create: NULL argument");
    *out = nullptr;
    const int nx = d->nx, ny = d->ny, nz = d->nz;
    if (nx < 8 || nx % 2 || !is_2a3b(nx / 2) || nx / 2 > 1024)
        return fail(FSEI_E_SHAPE, "nx = %d: need nx even, nx/2 = 2^a 3^b in [4, 1024]", nx);
    if (ny < 4 || ny % 2 || !is_2a3b(ny) || ny > 1024)
        return fail(FSEI_E_SHAPE, "ny = %d: need ny even, 2^a 3^b in [4, 1024]", ny);
    if (nz < 8 || nz > 2048) return fail(FSEI_E_SHAPE, "nz = %d: need 8 <= nz <= 2048", nz);
    if ((long long)nx * ny * nz > 0x7fffffffLL)
        return fail(FSEI_E_SHAPE, "%d x %d x %d cells: a field must hold fewer than 2^31 values", nx, ny, nz);
    if (!(d->lx > 0) || !(d->ly > 0)) return fail(FSEI_E_ARG, "lx, ly must be > 0");
    if (d->zbc != FSEI_Z_PERIODIC && d->zbc != FSEI_Z_WALLS) return fail(FSEI_E_ARG, "bad zbc %d", d->zbc);
    if (d->prec != FSEI_FP64 && d->prec != FSEI_MIXED) return fail(FSEI_E_ARG, "bad prec %d", d->prec);
    if (d->zbc == FSEI_Z_PERIODIC && !(d->lz > 0)) return fail(FSEI_E_ARG, "periodic z needs lz > 0");
    if (d->zbc == FSEI_Z_PERIODIC && d->zfaces) return fail(FSEI_E_ARG, "zfaces are for walls only");
    if (!(d->stretch >= 0)) return fail(FSEI_E_ARG, "stretch must be >= 0");

    // z faces (walls: tanh clustering on [-1, 1] or given faces)
    std::vector<double> zf(nz + 1);
    if (d->zbc == FSEI_Z_PERIODIC) {
        for (int k = 0; k <= nz; ++k) zf[k] = k * (d->lz / nz);
    } else if (d->zfaces) {
        for (int k = 0; k <= nz; ++k) zf[k] = d->zfaces[k];
        for (int k = 0; k < nz; ++k)
            if (!(zf[k + 1] > zf[k])) return fail(FSEI_E_ARG, "zfaces must increase strictly");
    } else if (d->stretch > 0) {
        const double s = d->stretch;
        for (int k = 0; k <= nz; ++k) zf[k] = tanh(s * (2.0 * k / nz - 1.0)) / tanh(s);
    } else {
        for (int k = 0; k <= nz; ++k) zf[k] = -1.0 + 2.0 * k / nz;
    }
    std::vector<double> dz(nz), idz(nz), hc(nz + 1), ihc(nz + 1);
    for (int k = 0; k < nz; ++k) dz[k] = zf[k + 1] - zf[k];
    for (int k = 1; k < nz; ++k) hc[k] = 0.5 * (zf[k + 1] + zf[k]) - 0.5 * (zf[k] + zf[k - 1]);
    if (d->zbc == FSEI_Z_WALLS) {
        hc[0] = 0.5 * dz[0];
        hc[nz] = 0.5 * dz[nz - 1];
    } else {
        hc[0] = hc[nz] = 0.5 * (dz[nz - 1] + dz[0]);
    }
    for (int k = 0; k < nz; ++k) idz[k] = 1.0 / dz[k];
    for (int k = 0; k <= nz; ++k) ihc[k] = 1.0 / hc[k];

    fsei_grid_s *G = new fsei_grid_s();
    G->desc = *d;
    G->desc.zfaces = nullptr;
    G->prec = d->prec;
    cudaGetDevice(&G->device);
    GridDev &g = G->g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.walls = d->zbc == FSEI_Z_WALLS;
    g.mx = nx / 2;
    g.sk = ((g.mx + 1 + 15) / 16) * 16;
    g.dx = d->lx / nx; g.dy = d->ly / ny;
    g.idx = 1.0 / g.dx; g.idy = 1.0 / g.dy;
    g.idx2 = g.idx * g.idx; g.idy2 = g.idy * g.idy;
    grid_float_copies(g);
    DevAllocs &M = G->mem;
    if (const char *cap = getenv("FSEI_WORKSPACE_LIMIT_BYTES")) {
        char *end = nullptr;
        const unsigned long long v = strtoull(cap, &end, 10);
        if (end != cap && *end == '\0') M.limit = (size_t)v;
    }
    if (const char *chk = getenv("FSEI_CHECK_BOUNDS")) M.guard = chk[0] != '\0' && chk[0] != '0';
    double *ddz = M.get<double>(nz), *didz = M.get<double>(nz), *dihc = M.get<double>(nz + 1);
    double *dzf = M.get<double>(nz + 1);
    float *fdz = M.get<float>(nz), *fidz = M.get<float>(nz), *fihc = M.get<float>(nz + 1);
    G->sc = M.get<StepScalars>(1);
    G->ib_count = M.get<int>(2);
    if (M.err != cudaSuccess) {
        M.release();
        delete G;
        return fail(FSEI_E_NOMEM, "metric allocation failed: %s", cudaGetErrorString(M.err));
    }
    auto tof = [](const std::vector<double> &v) {
        std::vector<float> o(v.size());
        for (size_t i = 0; i < v.size(); ++i) o[i] = (float)v[i];
        return o;
    };
    upload(ddz, dz); upload(didz, idz); upload(dihc, ihc); upload(dzf, zf);
    upload(fdz, tof(dz)); upload(fidz, tof(idz)); upload(fihc, tof(ihc));
    g.dz = ddz; g.idz = didz; g.ihc = dihc; g.zf = dzf;
    g.dzf = fdz; g.idzf = fidz; g.ihcf = fihc;
    cudaMemset(G->sc, 0, sizeof(StepScalars));
    if (cudaMallocHost((void **)&G->sc_host, sizeof(StepScalars)) != cudaSuccess) {
        M.release();
        delete G;
        return fail(FSEI_E_NOMEM, "pinned host allocation failed");
    }

    // modified wavenumbers and the modes solved exactly in double
    std::vector<double> lamx(g.sk), lamy(ny);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int kx = 0; kx < g.sk; ++kx)
        lamx[kx] = (double)((2.0L - 2.0L * cosl(2.0L * pi * kx / nx)) / ((long double)g.dx * g.dx));
    for (int ky = 0; ky < ny; ++ky)
        lamy[ky] = (double)((2.0L - 2.0L * cosl(2.0L * pi * ky / ny)) / ((long double)g.dy * g.dy));
    std::vector<int> nzm;
    nzm.push_back(0);
    if (d->prec == FSEI_MIXED) {
        const double tau = d->near_zero_tau > 0 ? d->near_zero_tau : 64.0;
        const double lz = zf[nz] - zf[0];
        for (int ky = 0; ky < ny; ++ky)
            for (int kx = 0; kx <= g.mx; ++kx) {
                if (kx == 0 && ky == 0) continue;
                if ((lamx[kx] + lamy[ky]) * lz * lz < tau) nzm.push_back(kx + g.sk * ky);
            }
    }
    fsei_status st = d->prec == FSEI_FP64
                         ? setup_work<double>(G, G->wd, lamx, lamy, nzm, dz, idz, ihc)
                         : setup_work<float>(G, G->wf, lamx, lamy, nzm, dz, idz, ihc);
    if (st == FSEI_OK) st = create_overlap(G);
    if (st == FSEI_OK) {
        Schedule cs;
        if (cached_schedule(G, &cs)) grid_apply(G, cs);
    }
    if (st != FSEI_OK) {
        destroy_overlap(G);
        cudaFreeHost(G->sc_host);
        M.release();
        delete G;
        return st;
    }
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        destroy_overlap(G);
        cudaFreeHost(G->sc_host);
        M.release();
        delete G;
        return fail(FSEI_E_CUDA, "grid setup: %s", cudaGetErrorString(e));
    }
    *out = G;
    return FSEI_OK;
}

void fsei_grid_destroy(fsei_grid G) {
    if (!G) return;
    DeviceGuard dg(G->device);
    cudaDeviceSynchronize();
    destroy_overlap(G);
    destroy_host_link(G);
    if (G->sc_host) cudaFreeHost(G->sc_host);
    G->mem.release();
    delete G;
    cudaGetLastError();   // teardown leaves no error behind for later calls
}

int64_t fsei_grid_workspace_bytes(fsei_grid G) { return G ? (int64_t)G->mem.bytes : 0; }

fsei_status fsei_grid_autotune(fsei_grid G, int32_t flags, void *cuda_stream, fsei_schedule *out) {
    NvtxRange nvtx_call("fsei_grid_autotune");
    g_err.clear();
    cudaGetLastError();
    if (!G) return fail(FSEI_E_ARG, "fsei_grid_autotune: NULL grid");
    if (flags & ~FSEI_TUNE_FORCE) return fail(FSEI_E_ARG, "fsei_grid_autotune: unknown flags %d", flags);
    DeviceGuard dg(G->device);
    Schedule cs;
    fsei_status r = FSEI_OK;
    if (!(flags & FSEI_TUNE_FORCE) && cached_schedule(G, &cs)) {
        grid_apply(G, cs);
    } else {
        cudaStream_t st = (cudaStream_t)cuda_stream;
        r = G->prec == FSEI_FP64 ? tune_grid<double>(G, G->wd, 8, st)
                                 : tune_grid<float>(G, G->wf, 8, st);
    }
    if (r == FSEI_OK && out) to_public(grid_schedule(G), out);
    return r;
}

fsei_status fsei_grid_get_schedule(fsei_grid G, fsei_schedule *out) {
    g_err.clear();
    if (!G || !out) return fail(FSEI_E_ARG, "fsei_grid_get_schedule: NULL argument");
    to_public(grid_schedule(G), out);
    return FSEI_OK;
}

fsei_status fsei_grid_set_schedule(fsei_grid G, const fsei_schedule *in) {
    g_err.clear();
    if (!G || !in) return fail(FSEI_E_ARG, "fsei_grid_set_schedule: NULL argument");
    Schedule s;
    s.rhs_cpl = in->rhs_cells_per_lane;
    s.rhs_strip = in->rhs_rows_per_strip;
    s.zsw_cols = in->zsweep_columns_per_lane;
    s.zl_lpl = in->poisson_lanes_per_line;
    s.zl_e = in->poisson_rows_per_lane;
    s.ry_rfft = in->rfft_rows_per_block;
    s.tkx_fft = in->ffty_columns_per_block;
    s.proj_mult = in->project_passes_per_thread;
    if (!schedule_valid(G, s))
        return fail(FSEI_E_ARG, "fsei_grid_set_schedule: a field is not a candidate of this grid");
    grid_apply(G, s);
    return FSEI_OK;
}

namespace {

// the checks fsei_step and fsei_step_host share: force alignment and the
// step parameters
fsei_status check_step_call(const void *fx, const void *fy, const void *fz,
                            const fsei_step_params *prm, int32_t nsteps, const char *who) {
    if (nsteps < 0) return fail(FSEI_E_ARG, "%s: nsteps < 0", who);
    const void *fo[3] = {fx, fy, fz};
    for (int i = 0; i < 3; ++i)
        if (fo[i] && !aligned16(fo[i])) return fail(FSEI_E_ARG, "force %d not 16-byte aligned", i);
    if (!(prm->re > 0)) return fail(FSEI_E_ARG, "re must be > 0");
    if (!(prm->cfl > 0) && !(prm->dt > 0)) return fail(FSEI_E_ARG, "need dt > 0 or cfl > 0");
    if (prm->scheme != FSEI_AB2_CN && prm->scheme != FSEI_RK3_CN)
        return fail(FSEI_E_ARG, "unknown scheme %d", prm->scheme);
    return check_rheology(*prm, who);
}

// synchronise st and fill the statistics of the last step; the status
// reports the device flags (non-finite first, then CFL)
fsei_status step_stats(fsei_grid_s *G, cudaStream_t st, fsei_step_stats *out, const char *who) {
    cudaMemcpyAsync(G->sc_host, G->sc, sizeof(StepScalars), cudaMemcpyDeviceToHost, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(FSEI_E_CUDA, "%s: %s", who, cudaGetErrorString(e));
    const StepScalars &h = *G->sc_host;
    out->dt_used = h.dt_step;
    const double spd = __builtin_bit_cast(double, h.speed_next);
    out->cfl = h.dt_step * spd;
    out->max_div = __builtin_bit_cast(double, h.maxdiv);
    out->kinetic_energy = h.ke;
    out->flags = h.flags;
    if (out->cfl > 1.0) out->flags |= FSEI_FLAG_CFL;
    if (out->flags & FSEI_FLAG_NONFINITE) return fail(FSEI_E_NONFINITE, "non-finite value in the new state");
    if (out->flags & FSEI_FLAG_CFL) return fail(FSEI_E_CFL, "CFL number %g above 1", out->cfl);
    return FSEI_OK;
}

// Bounds-checking mode: after the grid's work queued so far has finished,
// FSEI_E_BOUNDS if a guard zone of its workspace changed (FSEI_OK when the
// grid was created without guards).
fsei_status guard_status(const fsei_grid_s *G, const char *who) {
    if (!G->mem.guard) return FSEI_OK;
    size_t buf = 0, off = 0;
    int side = 0;
    cudaError_t e = cudaSuccess;
    if (G->mem.check_guards(&buf, &side, &off, &e))
        return fail(FSEI_E_BOUNDS,
                    "%s: the guard zone %s workspace buffer %zu (%zu bytes) was written %zu "
                    "bytes from the buffer's edge",
                    who, side ? "after" : "before", buf, G->mem.zones[buf].bytes, off);
    if (e != cudaSuccess) return fail(FSEI_E_CUDA, "%s: %s", who, cudaGetErrorString(e));
    return FSEI_OK;
}

// the status of a call that ran work on the grid, with the guard check of
// the bounds-checking mode taking precedence
fsei_status with_guards(const fsei_grid_s *G, fsei_status st, const char *who) {
    if (!G->mem.guard) return st;
    const fsei_status g = guard_status(G, who);
    return g != FSEI_OK ? g : st;
}

}  // namespace

fsei_status fsei_step(fsei_grid G, fsei_state *s, const void *fx, const void *fy, const void *fz,
                      const fsei_step_params *prm, int32_t nsteps, void *cuda_stream,
                      fsei_step_stats *out) {
    NvtxRange nvtx_call("fsei_step");
    g_err.clear();
    cudaGetLastError();   // an error left by an unrelated earlier call is not ours
    if (!G || !s || !prm) return fail(FSEI_E_ARG, "fsei_step: NULL argument");
    const void *req[7] = {s->u, s->v, s->w, s->p, s->hu, s->hv, s->hw};
    for (int i = 0; i < 7; ++i) {
        if (!req[i]) return fail(FSEI_E_ARG, "state field %d is NULL", i);
        if (!aligned16(req[i])) return fail(FSEI_E_ARG, "state field %d not 16-byte aligned", i);
    }
    {
        const fsei_status rs = check_step_call(fx, fy, fz, prm, nsteps, "fsei_step");
        if (rs != FSEI_OK) return rs;
    }
    const StepArgs a = step_args(*prm);
    DeviceGuard dg(G->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    fsei_status r = FSEI_OK;
    if (nsteps > 0) {
        r = G->prec == FSEI_FP64 ? run_steps<double>(G, G->wd, s, fx, fy, fz, a, nsteps, st)
                                 : run_steps<float>(G, G->wf, s, fx, fy, fz, a, nsteps, st);
        if (r != FSEI_OK) return r;
        s->have_prev_h = 1;
    }
    return with_guards(G, out ? step_stats(G, st, out, "fsei_step") : FSEI_OK, "fsei_step");
}

fsei_status fsei_step_host(fsei_grid G, fsei_state *host, const fsei_state *dev, const void *fx,
                           const void *fy, const void *fz, const fsei_step_params *prm,
                           int32_t nsteps, void *cuda_stream, fsei_step_stats *out) {
    NvtxRange nvtx_call("fsei_step_host");
    g_err.clear();
    cudaGetLastError();
    if (!G || !host || !dev || !prm) return fail(FSEI_E_ARG, "fsei_step_host: NULL argument");
    void *hf[7] = {host->u, host->v, host->w, host->p, host->hu, host->hv, host->hw};
    void *df[7] = {dev->u, dev->v, dev->w, dev->p, dev->hu, dev->hv, dev->hw};
    for (int i = 0; i < 7; ++i) {
        if (!hf[i]) return fail(FSEI_E_ARG, "host field %d is NULL", i);
        if (!df[i]) return fail(FSEI_E_ARG, "device field %d is NULL", i);
        if (!aligned16(df[i])) return fail(FSEI_E_ARG, "device field %d not 16-byte aligned", i);
    }
    {
        const fsei_status rs = check_step_call(fx, fy, fz, prm, nsteps, "fsei_step_host");
        if (rs != FSEI_OK) return rs;
    }
    const StepArgs a = step_args(*prm);
    DeviceGuard dg(G->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    {
        const fsei_status rs = create_host_link(G);
        if (rs != FSEI_OK) return rs;
    }
    auto &H = G->host;
    const size_t bytes = (size_t)G->g.nx * G->g.ny * G->g.nz * (G->prec == FSEI_FP64 ? 8 : 4);
    // in: after the work queued on st so far (the device buffers are free),
    // the history fields first (their copies back from the previous call
    // land first), each field after its own copy back
    cudaEventRecord(H.entry, st);
    cudaStreamWaitEvent(H.h2d, H.entry, 0);
    const int in_order[7] = {4, 5, 6, 0, 1, 2, 3};
    for (int f : in_order) {
        if (H.back_valid) cudaStreamWaitEvent(H.h2d, H.back[f], 0);
        cudaMemcpyAsync(df[f], hf[f], bytes, cudaMemcpyHostToDevice, H.h2d);
    }
    cudaEventRecord(H.in, H.h2d);
    cudaStreamWaitEvent(st, H.in, 0);
    fsei_state ds = *dev;
    ds.have_prev_h = host->have_prev_h;
    if (nsteps > 0) {
        const fsei_status r =
            G->prec == FSEI_FP64
                ? run_steps<double>(G, G->wd, &ds, fx, fy, fz, a, nsteps, st, true, H.rhs)
                : run_steps<float>(G, G->wf, &ds, fx, fy, fz, a, nsteps, st, true, H.rhs);
        if (r != FSEI_OK) return r;
        host->have_prev_h = 1;
    }
    cudaEventRecord(H.step, st);
    // out: H^n once the last right-hand side has written it (under the rest
    // of the step), then u, v, w, p after the step
    cudaStreamWaitEvent(H.d2h, nsteps > 0 ? H.rhs : H.step, 0);
    for (int f = 4; f < 7; ++f) {
        cudaMemcpyAsync(hf[f], df[f], bytes, cudaMemcpyDeviceToHost, H.d2h);
        cudaEventRecord(H.back[f], H.d2h);
    }
    cudaStreamWaitEvent(H.d2h, H.step, 0);
    for (int f = 0; f < 4; ++f) {
        cudaMemcpyAsync(hf[f], df[f], bytes, cudaMemcpyDeviceToHost, H.d2h);
        cudaEventRecord(H.back[f], H.d2h);
    }
    H.back_valid = true;
    cudaEventRecord(H.out, H.d2h);
    H.out_valid = true;
    if (out) cudaStreamWaitEvent(st, H.out, 0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FSEI_E_CUDA, "fsei_step_host: %s", cudaGetErrorString(e));
    return with_guards(G, out ? step_stats(G, st, out, "fsei_step_host") : FSEI_OK,
                       "fsei_step_host");
}

fsei_status fsei_step_host_join(fsei_grid G, void *cuda_stream) {
    g_err.clear();
    if (!G) return fail(FSEI_E_ARG, "fsei_step_host_join: NULL grid");
    DeviceGuard dg(G->device);
    if (G->host.out_valid) cudaStreamWaitEvent((cudaStream_t)cuda_stream, G->host.out, 0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FSEI_E_CUDA, "fsei_step_host_join: %s", cudaGetErrorString(e));
    return FSEI_OK;
}

fsei_status fsei_adjoint_step(fsei_grid G, const fsei_state *fwd, const fsei_step_params *prm,
                              fsei_state *adj, void *fbar_x, void *fbar_y, void *fbar_z,
                              void *cuda_stream) {
    NvtxRange nvtx_call("fsei_adjoint_step");
    g_err.clear();
    cudaGetLastError();   // an error left by an unrelated earlier call is not ours
    if (!G || !fwd || !prm || !adj) return fail(FSEI_E_ARG, "fsei_adjoint_step: NULL argument");
    const void *fw[3] = {fwd->u, fwd->v, fwd->w};
    for (int i = 0; i < 3; ++i)
        if (!fw[i] || !aligned16(fw[i])) return fail(FSEI_E_ARG, "forward field %d NULL or misaligned", i);
    const void *ad[7] = {adj->u, adj->v, adj->w, adj->p, adj->hu, adj->hv, adj->hw};
    for (int i = 0; i < 7; ++i)
        if (!ad[i] || !aligned16(ad[i])) return fail(FSEI_E_ARG, "cotangent field %d NULL or misaligned", i);
    const void *fb[3] = {fbar_x, fbar_y, fbar_z};
    for (int i = 0; i < 3; ++i)
        if (fb[i] && !aligned16(fb[i])) return fail(FSEI_E_ARG, "fbar %d not 16-byte aligned", i);
    if (!(prm->re > 0)) return fail(FSEI_E_ARG, "re must be > 0");
    if (prm->cfl > 0) return fail(FSEI_E_ARG, "the adjoint needs a frozen dt: pass cfl = 0 and the dt of the forward step");
    if (!(prm->dt > 0)) return fail(FSEI_E_ARG, "dt must be > 0");
    if (prm->scheme != FSEI_AB2_CN)
        return fail(prm->scheme == FSEI_RK3_CN ? FSEI_E_UNSUPPORTED : FSEI_E_ARG,
                    "the adjoint step is implemented for the Adams-Bashforth scheme only");
    if (prm->rheology != FSEI_NEWTONIAN)
        return fail(FSEI_E_UNSUPPORTED, "the adjoint step is implemented for the Newtonian stress only");
    StepArgs a = step_args(*prm);
    a.cfl = 0.0;
    DeviceGuard dg(G->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    auto run = [&](auto &W, auto tag) -> fsei_status {
        using T = decltype(tag);
        const size_t ncell = (size_t)G->g.nx * G->g.ny * G->g.nz;
        if (!W.adj0) {
            W.adj0 = G->mem.get<T>(ncell);
            W.adj1 = G->mem.get<T>(ncell);
            W.adj2 = G->mem.get<T>(ncell);
            if (G->mem.err != cudaSuccess) {
                W.adj0 = W.adj1 = W.adj2 = nullptr;
                G->mem.err = cudaSuccess;
                return fail(FSEI_E_NOMEM, "adjoint workspace allocation failed");
            }
        }
        const int euler = fwd->have_prev_h ? 0 : 1;
        KernelTimer &tm = G->timer;
        tm.run(KK_BEGIN, st, [&] { launch_step_begin<T>(G->g, W, G->sc, a, euler, st); });
        LaunchHook hook;
        hook.ctx = &tm;
        hook.before = [](void *c, int kind, cudaStream_t s2) {
            static_cast<KernelTimer *>(c)->begin(KK_ADJ_FIRST + kind, s2);
        };
        hook.after = [](void *c, int, cudaStream_t s2) { static_cast<KernelTimer *>(c)->end(s2); };
        launch_adjoint_step<T>(G->g, W, G->sc, (const T *)fwd->u, (const T *)fwd->v,
                               (const T *)fwd->w, (T *)adj->u, (T *)adj->v, (T *)adj->w,
                               (T *)adj->p, (T *)adj->hu, (T *)adj->hv, (T *)adj->hw,
                               (T *)fbar_x, (T *)fbar_y, (T *)fbar_z, prm->re, st,
                               &hook);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(FSEI_E_CUDA, "adjoint launch: %s", cudaGetErrorString(e));
        return FSEI_OK;
    };
    return with_guards(G, G->prec == FSEI_FP64 ? run(G->wd, double(0)) : run(G->wf, float(0)),
                       "fsei_adjoint_step");
}

fsei_status fsei_poisson_solve(fsei_grid G, const void *rhs, void *phi, void *cuda_stream) {
    NvtxRange nvtx_call("fsei_poisson_solve");
    g_err.clear();
    cudaGetLastError();   // an error left by an unrelated earlier call is not ours
    if (!G || !rhs || !phi) return fail(FSEI_E_ARG, "fsei_poisson_solve: NULL argument");
    if (!aligned16(rhs) || !aligned16(phi)) return fail(FSEI_E_ARG, "rhs/phi not 16-byte aligned");
    DeviceGuard dg(G->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    return with_guards(G,
                       G->prec == FSEI_FP64 ? run_poisson<double>(G, G->wd, rhs, phi, st)
                                            : run_poisson<float>(G, G->wf, rhs, phi, st),
                       "fsei_poisson_solve");
}

// the launch check and skipped-count read-back of the two IB entry points
static fsei_status ib_finish(fsei_grid_s *G, cudaStream_t st, int32_t *skipped, int count,
                      const char *what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FSEI_E_CUDA, "%s launch: %s", what, cudaGetErrorString(e));
    if (skipped) {
        int h[2] = {0, 0};
        if (cudaMemcpyAsync(h, G->ib_count, sizeof(int) * count, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return fail(FSEI_E_CUDA, "%s: read-back failed", what);
        for (int i = 0; i < count; ++i) skipped[i] = h[i];
    }
    return FSEI_OK;
}

fsei_status fsei_ib_forcing(fsei_grid G, const void *u, const void *v, const void *w,
                            const double *xb, const double *ub, const double *dvb,
                            int32_t nmarkers, double dt, void *fx, void *fy, void *fz,
                            double *u_at, void *cuda_stream, int32_t *skipped) {
    NvtxRange nvtx_call("fsei_ib_forcing");
    g_err.clear();
    cudaGetLastError();
    if (!G || !u || !v || !w || !fx || !fy || !fz) return fail(FSEI_E_ARG, "fsei_ib_forcing: NULL argument");
    if (nmarkers < 0 || (nmarkers > 0 && (!xb || !ub || !dvb)))
        return fail(FSEI_E_ARG, "fsei_ib_forcing: bad marker arrays");
    if (nmarkers > (1 << 29)) return fail(FSEI_E_ARG, "fsei_ib_forcing: too many markers");
    if (!(dt > 0)) return fail(FSEI_E_ARG, "fsei_ib_forcing: dt must be > 0");
    DeviceGuard dg(G->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaMemsetAsync(G->ib_count, 0, sizeof(int), st);
    if (G->prec == FSEI_FP64)
        launch_ib_force<double>(G->g, (const double *)u, (const double *)v, (const double *)w, xb,
                                ub, dvb, nmarkers, dt, (double *)fx, (double *)fy, (double *)fz,
                                u_at, G->ib_count, st);
    else
        launch_ib_force<float>(G->g, (const float *)u, (const float *)v, (const float *)w, xb, ub,
                               dvb, nmarkers, dt, (float *)fx, (float *)fy, (float *)fz, u_at,
                               G->ib_count, st);
    return with_guards(G, ib_finish(G, st, skipped, 1, "fsei_ib_forcing"), "fsei_ib_forcing");
}

fsei_status fsei_ib_loads(fsei_grid G, const void *p, const void *u, const void *v,
                          const void *w, const double *xf, const double *nf, const double *af,
                          const int32_t *two_sided, const int32_t *tris, int32_t nfaces,
                          int32_t nnodes, double probe, double re, double *face_force,
                          double *node_force, void *cuda_stream, int32_t *skipped) {
    NvtxRange nvtx_call("fsei_ib_loads");
    g_err.clear();
    cudaGetLastError();
    if (!G || !p || !u || !v || !w) return fail(FSEI_E_ARG, "fsei_ib_loads: NULL field");
    if (nfaces < 0 || (nfaces > 0 && (!xf || !nf || !af || !face_force)))
        return fail(FSEI_E_ARG, "fsei_ib_loads: bad face arrays");
    if (nfaces > (1 << 26)) return fail(FSEI_E_ARG, "fsei_ib_loads: too many faces");
    if (node_force && (!tris || nnodes < 1))
        return fail(FSEI_E_ARG, "fsei_ib_loads: nodal loads need tris and nnodes >= 1");
    if (!(probe > 0) || !(re > 0)) return fail(FSEI_E_ARG, "fsei_ib_loads: probe and re must be > 0");
    DeviceGuard dg(G->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaMemsetAsync(G->ib_count, 0, 2 * sizeof(int), st);
    if (G->prec == FSEI_FP64)
        launch_ib_loads<double>(G->g, (const double *)p, (const double *)u, (const double *)v,
                                (const double *)w, xf, nf, af, two_sided, tris, nfaces, nnodes,
                                probe, 1.0 / re, face_force, node_force, G->ib_count, st);
    else
        launch_ib_loads<float>(G->g, (const float *)p, (const float *)u, (const float *)v,
                               (const float *)w, xf, nf, af, two_sided, tris, nfaces, nnodes,
                               probe, 1.0 / re, face_force, node_force, G->ib_count, st);
    return with_guards(G, ib_finish(G, st, skipped, 2, "fsei_ib_loads"), "fsei_ib_loads");
}

fsei_status fsei_grid_check_bounds(fsei_grid G) {
    g_err.clear();
    if (!G) return fail(FSEI_E_ARG, "fsei_grid_check_bounds: NULL grid");
    if (!G->mem.guard)
        return fail(FSEI_E_UNSUPPORTED, "the grid was created without FSEI_CHECK_BOUNDS=1");
    DeviceGuard dg(G->device);
    return guard_status(G, "fsei_grid_check_bounds");
}

fsei_status fsei_grid_poke_guard(fsei_grid G, int32_t buffer, int32_t side, int64_t offset) {
    g_err.clear();
    if (!G) return fail(FSEI_E_ARG, "fsei_grid_poke_guard: NULL grid");
    if (!G->mem.guard)
        return fail(FSEI_E_UNSUPPORTED, "the grid was created without FSEI_CHECK_BOUNDS=1");
    if (buffer < 0 || (size_t)buffer >= G->mem.zones.size() || (side != 0 && side != 1))
        return fail(FSEI_E_ARG, "fsei_grid_poke_guard: no guard zone %d/%d", buffer, side);
    const DevAllocs::Zone &z = G->mem.zones[(size_t)buffer];
    if (offset < 0 || (size_t)offset >= z.gbytes)
        return fail(FSEI_E_ARG, "fsei_grid_poke_guard: offset %lld outside the zone",
                    (long long)offset);
    DeviceGuard dg(G->device);
    // the byte `offset` bytes from the buffer's edge, inside the zone
    const unsigned char *p = side ? z.back + offset : z.front + (z.gbytes - 1 - (size_t)offset);
    const cudaError_t e = cudaMemset(const_cast<unsigned char *>(p), z.fill ^ 0x5A, 1);
    if (e == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess) return FSEI_OK;
    return fail(FSEI_E_CUDA, "fsei_grid_poke_guard: %s", cudaGetErrorString(cudaGetLastError()));
}

fsei_status fsei_set_kernel_timing(fsei_grid G, int32_t enable) {
    g_err.clear();
    if (!G) return fail(FSEI_E_ARG, "fsei_set_kernel_timing: NULL grid");
    DeviceGuard dg(G->device);
    if (!enable) G->timer.collect();
    G->timer.on = enable != 0;
    return FSEI_OK;
}

int32_t fsei_kernel_times(fsei_grid G, double *total_ms, int64_t *launches, int32_t cap) {
    if (!G) return 0;
    DeviceGuard dg(G->device);
    G->timer.collect();
    for (int k = 0; k < KK_COUNT && k < cap; ++k) {
        if (total_ms) total_ms[k] = G->timer.ms[k];
        if (launches) launches[k] = G->timer.n[k];
    }
    for (int k = 0; k < KK_COUNT; ++k) {
        G->timer.ms[k] = 0;
        G->timer.n[k] = 0;
    }
    return KK_COUNT;
}

const char *fsei_kernel_name(int32_t kind) {
    return (kind >= 0 && kind < KK_COUNT) ? kKernelNames[kind] : nullptr;
}

}  // extern "C"

// ------------------------------------------------------------- batches ----
// An ensemble of independent grids advanced together.  Boxes with the same
// grid description (extents, lengths, z mesh, precision) and launch schedule
// form a group: every pass of the step (scalars, z-sweep plans, RHS + x
// sweep, y and z sweeps, the transforms and z Poisson solve, the projection)
// is one launch over all boxes of the group, box b in blockIdx.z with its own
// arguments (fields, workspace, step parameters) from a table passed as the
// launch's parameter.  One
// step of every group is captured into a CUDA graph, the groups on parallel
// branches, and the graph is replayed once per step on the caller's stream.
// Two graphs are kept: the first step of a call (CFL pre-pass, Euler start
// for boxes without history) and the following steps.  They are re-captured
// when the state pointers, forces or parameters of a call differ from the
// captured ones.
// Boxes per launch group by default (0: every box of a description in one
// launch group).  Smaller launch groups on parallel branches let the passes
// of different groups run side by side; measured on the 64-box ensemble of
// four shapes, one launch group per shape was the fastest (15.4 Gcell/s,
// against 14.6 with one box per launch group).
constexpr int kDefaultMaxGroup = 0;

struct fsei_batch_s {
    std::vector<fsei_grid> grids;
    std::vector<std::vector<unsigned char>> desc_key;   // per box: its description
    int device = 0;
    std::vector<cudaStream_t> branches;
    cudaStream_t capture = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> joins;
    cudaGraphExec_t first = nullptr, rest = nullptr;
    std::vector<unsigned char> key;   // bytes of the captured call's arguments
    int ngroups = 0;                  // launch groups of the last capture
    int max_group = kDefaultMaxGroup; // boxes per launch group (0: no limit)
};

namespace {

void batch_clear_graphs(fsei_batch_s *B) {
    if (B->first) cudaGraphExecDestroy(B->first);
    if (B->rest) cudaGraphExecDestroy(B->rest);
    B->first = B->rest = nullptr;
    B->key.clear();
}

template <typename X> void put_bytes(std::vector<unsigned char> &v, const X &x) {
    const unsigned char *c = reinterpret_cast<const unsigned char *>(&x);
    v.insert(v.end(), c, c + sizeof(X));
}

// the description of a box as bytes (faces copied when given)
std::vector<unsigned char> desc_bytes(const fsei_grid_desc &d) {
    std::vector<unsigned char> k;
    put_bytes(k, d.nx); put_bytes(k, d.ny); put_bytes(k, d.nz);
    put_bytes(k, d.lx); put_bytes(k, d.ly); put_bytes(k, d.zbc); put_bytes(k, d.lz);
    put_bytes(k, d.stretch); put_bytes(k, d.prec); put_bytes(k, d.near_zero_tau);
    const int has = d.zfaces ? 1 : 0;
    put_bytes(k, has);
    if (has)
        for (int i = 0; i <= d.nz; ++i) put_bytes(k, d.zfaces[i]);
    return k;
}

// two recorded steps launch the same kernels with the same shapes
bool same_launches(const std::vector<RecordedOp> &a, const std::vector<RecordedOp> &b,
                   cudaStream_t side_a, cudaStream_t side_b) {
    if (a.size() != b.size()) return false;
    for (size_t i = 0; i < a.size(); ++i) {
        const RecordedOp &x = a[i], &y = b[i];
        if (x.kind != y.kind || (x.st == side_a) != (y.st == side_b)) return false;
        if (x.kind == RecordedOp::KERNEL &&
            (x.entry != y.entry || x.grid.x != y.grid.x || x.grid.y != y.grid.y ||
             x.block.x != y.block.x || x.block.y != y.block.y || x.block.z != y.block.z ||
             x.smem != y.smem || x.pdl != y.pdl || x.args.size() != y.args.size()))
            return false;
        if (x.kind == RecordedOp::MEMSET && x.mem_bytes != y.mem_bytes) return false;
    }
    return true;
}

fsei_status batch_capture(fsei_batch_s *B, fsei_state *states, const void *const *forces,
                          const fsei_step_params *prm, bool first, cudaGraphExec_t *out) {
    const size_t nb = B->grids.size();
    // 1. one recorded step per box (nothing is launched)
    std::vector<std::vector<RecordedOp>> rec(nb);
    const cudaStream_t main_tag = B->capture;   // stands for the box's main stream
    for (size_t i = 0; i < nb; ++i) {
        fsei_grid_s *G = B->grids[i];
        const StepArgs a = step_args(prm[i]);
        fsei_state s = states[i];
        if (!first) s.have_prev_h = 1;
        const void *f0 = forces ? forces[3 * i] : nullptr;
        const void *f1 = forces ? forces[3 * i + 1] : nullptr;
        const void *f2 = forces ? forces[3 * i + 2] : nullptr;
        LaunchRecorder r;
        launch_recorder() = &r;
        const bool timing = G->timer.on;
        G->timer.on = false;
        const fsei_status st = G->prec == FSEI_FP64
                                   ? run_steps<double>(G, G->wd, &s, f0, f1, f2, a, 1, main_tag, first)
                                   : run_steps<float>(G, G->wf, &s, f0, f1, f2, a, 1, main_tag, first);
        G->timer.on = timing;
        launch_recorder() = nullptr;
        if (st != FSEI_OK) {
            const std::string msg = g_err;
            return fail(st, "batch: box %zu: %s", i, msg.c_str());
        }
        rec[i] = std::move(r.ops);
    }
    // 2. groups: same description, schedule and launch sequence
    std::vector<std::vector<size_t>> groups;
    std::vector<std::vector<unsigned char>> gkeys;
    for (size_t i = 0; i < nb; ++i) {
        std::vector<unsigned char> k = B->desc_key[i];
        put_bytes(k, grid_schedule(B->grids[i]));
        size_t gi = 0;
        for (; gi < groups.size(); ++gi) {
            const size_t b0 = groups[gi][0];
            if (gkeys[gi] == k && same_launches(rec[b0], rec[i], B->grids[b0]->ov_plans.side,
                                                B->grids[i]->ov_plans.side))
                break;
        }
        if (gi == groups.size()) {
            groups.emplace_back();
            gkeys.push_back(k);
        }
        groups[gi].push_back(i);
    }
    // at most max_group boxes per launch group, and no more than the
    // argument-table capacity of any of the group's kernels
    {
        std::vector<std::vector<size_t>> split;
        for (const std::vector<size_t> &g : groups) {
            size_t cap = B->max_group > 0 ? (size_t)B->max_group : g.size();
            for (const RecordedOp &op : rec[g[0]])
                if (op.kind == RecordedOp::KERNEL) cap = std::min(cap, (size_t)op.group_cap);
            for (size_t a = 0; a < g.size(); a += cap)
                split.emplace_back(g.begin() + a, g.begin() + std::min(g.size(), a + cap));
        }
        groups.swap(split);
    }
    // 3. argument rows: for every kernel of a launch group, the boxes'
    // argument tuples back to back (they become the launch's parameter)
    std::vector<std::vector<std::vector<unsigned char>>> rows(groups.size());
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        const std::vector<RecordedOp> &ops = rec[groups[gi][0]];
        rows[gi].resize(ops.size());
        for (size_t o = 0; o < ops.size(); ++o) {
            if (ops[o].kind != RecordedOp::KERNEL) continue;
            for (size_t b : groups[gi])
                rows[gi][o].insert(rows[gi][o].end(), rec[b][o].args.begin(), rec[b][o].args.end());
            ops[o].prepare_group();   // load it outside the capture
        }
    }
    // 4. capture: every group on a branch, its side stream for the plans
    cudaStream_t cs = B->capture;
    cudaGetLastError();
    cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (ce != cudaSuccess)
        return fail(FSEI_E_CUDA, "batch: cannot begin graph capture: %s", cudaGetErrorString(ce));
    ce = cudaEventRecord(B->fork, cs);
    for (cudaStream_t b : B->branches)
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b, B->fork, 0);
    fsei_status r = ce == cudaSuccess ? FSEI_OK
                                      : fail(FSEI_E_CUDA, "batch: fork: %s", cudaGetErrorString(ce));
    for (size_t gi = 0; gi < groups.size() && r == FSEI_OK; ++gi) {
        const std::vector<size_t> &bx = groups[gi];
        fsei_grid_s *G0 = B->grids[bx[0]];
        const Overlap &ov = G0->ov_plans;
        const cudaStream_t mst = B->branches[gi % B->branches.size()];
        const std::vector<RecordedOp> &ops = rec[bx[0]];
        for (size_t o = 0; o < ops.size() && r == FSEI_OK; ++o) {
            const RecordedOp &op = ops[o];
            const cudaStream_t st = op.st == ov.side ? ov.side : mst;
            switch (op.kind) {
            case RecordedOp::KERNEL:
                op.launch_group(rows[gi][o].data(), (int)bx.size(), op.grid, op.block, op.smem, st,
                                op.pdl);
                break;
            case RecordedOp::MEMSET:
                for (size_t b : bx) cudaMemsetAsync(rec[b][o].mem, 0, rec[b][o].mem_bytes, st);
                break;
            case RecordedOp::FORK:
                cudaEventRecord(ov.fork, mst);
                cudaStreamWaitEvent(ov.side, ov.fork, 0);
                break;
            case RecordedOp::JOIN:
                cudaEventRecord(ov.join, ov.side);
                cudaStreamWaitEvent(mst, ov.join, 0);
                break;
            }
            const cudaError_t e = cudaPeekAtLastError();
            if (e != cudaSuccess)
                r = fail(FSEI_E_CUDA, "batch capture, group %zu (%zu boxes from box %zu), launch %zu: %s",
                         gi, bx.size(), bx[0], o, cudaGetErrorString(e));
        }
    }
    for (size_t b = 0; b < B->branches.size(); ++b) {
        cudaEventRecord(B->joins[b], B->branches[b]);
        cudaStreamWaitEvent(cs, B->joins[b], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (r == FSEI_OK && (e != cudaSuccess || !graph))
        r = fail(FSEI_E_CUDA, "batch: capture failed: %s", cudaGetErrorString(e));
    if (r == FSEI_OK) {
        const cudaError_t ei = cudaGraphInstantiate(out, graph, 0);
        if (ei != cudaSuccess)
            r = fail(FSEI_E_CUDA, "batch: graph instantiation failed: %s", cudaGetErrorString(ei));
    }
    if (graph) cudaGraphDestroy(graph);
    if (r != FSEI_OK) {
        cudaGetLastError();
        return r;
    }
    B->ngroups = (int)groups.size();
    return FSEI_OK;
}

// Refine the schedule of the boxes idx (one shape, two or more boxes) by
// timing their grouped launches: knob by knob, every candidate applied to
// all of them, one step of the group captured into a graph on stand-in
// fields and replayed; the median replay time decides (a challenger must
// be 0.5 % faster).  A solo grid of a shape tunes each kernel for a launch
// of that grid alone; in a group every launch covers all boxes, which
// moves the best tile shapes (more rows per block pay once the blocks of
// many boxes fill the GPU).  Skipped, not failed, when the stand-in fields
// do not fit.
std::mutex g_group_mu;
std::vector<std::pair<ScheduleKey, size_t>> g_group_tuned;   // (shape, boxes) measured

fsei_status tune_group(fsei_batch_s *B, const std::vector<size_t> &idx, cudaStream_t st,
                       bool force) {
    fsei_grid_s *G0 = B->grids[idx[0]];
    const std::pair<ScheduleKey, size_t> gk(schedule_key(G0), idx.size());
    {
        std::lock_guard<std::mutex> lk(g_group_mu);
        const bool seen = std::find(g_group_tuned.begin(), g_group_tuned.end(), gk) != g_group_tuned.end();
        if (seen && !force) return FSEI_OK;   // the cached schedule is the group's
        if (!seen) g_group_tuned.push_back(gk);
    }
    const size_t ncell = (size_t)G0->g.nx * G0->g.ny * G0->g.nz;
    const size_t esz = G0->prec == FSEI_FP64 ? 8 : 4;
    std::vector<void *> bufs;
    std::vector<fsei_state> states(idx.size());
    bool fits = true;
    for (size_t b = 0; b < idx.size() && fits; ++b) {
        void *p = nullptr;
        fits = cudaMalloc(&p, 7 * ncell * esz) == cudaSuccess;
        if (!fits) break;
        bufs.push_back(p);
        cudaMemsetAsync(p, 0x3c, 7 * ncell * esz, st);
        unsigned char *c = static_cast<unsigned char *>(p);
        fsei_state &s = states[b];
        s.u = c; s.v = c + ncell * esz; s.w = c + 2 * ncell * esz; s.p = c + 3 * ncell * esz;
        s.hu = c + 4 * ncell * esz; s.hv = c + 5 * ncell * esz; s.hw = c + 6 * ncell * esz;
        s.have_prev_h = 1;
    }
    auto release = [&] {
        cudaStreamSynchronize(st);
        for (void *p : bufs) cudaFree(p);
        cudaGetLastError();
    };
    if (!fits) {
        release();
        return FSEI_OK;
    }
    // a view of the shape's boxes on the batch's capture stream and first
    // branch (it owns nothing: never passed to fsei_batch_destroy)
    fsei_batch_s sub;
    sub.device = B->device;
    for (size_t b : idx) {
        sub.grids.push_back(B->grids[b]);
        sub.desc_key.push_back(B->desc_key[b]);
    }
    sub.branches.assign(1, B->branches[0]);
    sub.joins.assign(1, B->joins[0]);
    sub.capture = B->capture;
    sub.fork = B->fork;
    sub.max_group = B->max_group;
    fsei_step_params tp = {};
    tp.re = 1000.0; tp.dt = 1e-4; tp.gamma = 1.5; tp.rho = -0.5;
    std::vector<fsei_step_params> prm(idx.size(), tp);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // median device time of one replayed step of the group with schedule s;
    // < 0 where the group cannot be captured with it
    auto trial = [&](const Schedule &sch) -> double {
        for (fsei_grid_s *G : sub.grids) grid_apply(G, sch);
        cudaGraphExec_t ge = nullptr;
        if (batch_capture(&sub, states.data(), nullptr, prm.data(), false, &ge) != FSEI_OK) {
            g_err.clear();
            cudaGetLastError();
            return -1.0;
        }
        cudaGraphLaunch(ge, st);
        float t[7];
        for (int r = 0; r < 7; ++r) {
            cudaEventRecord(e0, st);
            cudaGraphLaunch(ge, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            t[r] = 0.0f;
            cudaEventElapsedTime(&t[r], e0, e1);
        }
        cudaGraphExecDestroy(ge);
        std::sort(t, t + 7);
        return cudaGetLastError() == cudaSuccess ? (double)t[3] : -1.0;
    };
    Schedule cur = grid_schedule(G0);
    for (int knob = 0; knob < SK_COUNT; ++knob) {
        int cand[16][2];
        const int nc = G0->prec == FSEI_FP64 ? schedule_candidates<double>(G0->g, knob, cand, 16)
                                             : schedule_candidates<float>(G0->g, knob, cand, 16);
        if (nc < 2) continue;
        double best_ms = trial(cur);
        for (int c = 0; c < nc; ++c) {
            Schedule s = cur;
            set_knob(s, knob, cand[c]);
            if (memcmp(&s, &cur, sizeof s) == 0) continue;
            const double t = trial(s);
            if (t > 0.0 && (best_ms <= 0.0 || t < 0.995 * best_ms)) {
                best_ms = t;
                cur = s;
            }
        }
    }
    for (fsei_grid_s *G : sub.grids) grid_apply(G, cur);
    store_schedule(G0, cur);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release();
    sub.grids.clear();
    return FSEI_OK;
}

}  // namespace

extern "C" {

fsei_status fsei_batch_create(const fsei_grid_desc *descs, int32_t nboxes, fsei_batch *out) {
    NvtxRange nvtx_call("fsei_batch_create");
    g_err.clear();
    if (!descs || !out || nboxes < 1) return fail(FSEI_E_ARG, "fsei_batch_create: bad arguments");
    *out = nullptr;
    fsei_batch_s *B = new fsei_batch_s();
    cudaGetDevice(&B->device);
    for (int i = 0; i < nboxes; ++i) {
        fsei_grid g = nullptr;
        const fsei_status st = fsei_grid_create(&descs[i], &g);
        if (st != FSEI_OK) {
            const std::string msg = g_err;
            fsei_batch_destroy(B);
            return fail(st, "box %d: %s", i, msg.c_str());
        }
        B->grids.push_back(g);
        B->desc_key.push_back(desc_bytes(descs[i]));
    }
    const int nb = nboxes < 8 ? nboxes : 8;
    B->branches.resize(nb);
    B->joins.resize(nb);
    bool ok = cudaStreamCreateWithFlags(&B->capture, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int b = 0; b < nb && ok; ++b)
        ok = cudaStreamCreateWithFlags(&B->branches[b], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&B->joins[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        fsei_batch_destroy(B);
        return fail(FSEI_E_CUDA, "fsei_batch_create: stream/event creation failed");
    }
    *out = B;
    return FSEI_OK;
}

void fsei_batch_destroy(fsei_batch B) {
    if (!B) return;
    DeviceGuard dg(B->device);
    cudaDeviceSynchronize();
    batch_clear_graphs(B);
    for (cudaStream_t s : B->branches)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : B->joins)
        if (e) cudaEventDestroy(e);
    if (B->capture) cudaStreamDestroy(B->capture);
    if (B->fork) cudaEventDestroy(B->fork);
    for (fsei_grid g : B->grids) fsei_grid_destroy(g);
    delete B;
    cudaGetLastError();
}

int32_t fsei_batch_size(fsei_batch B) { return B ? (int32_t)B->grids.size() : 0; }

fsei_status fsei_batch_set_max_group(fsei_batch B, int32_t max_boxes) {
    g_err.clear();
    if (!B) return fail(FSEI_E_ARG, "fsei_batch_set_max_group: NULL batch");
    if (max_boxes < 0) return fail(FSEI_E_ARG, "max_boxes must be >= 0");
    if (max_boxes != B->max_group) {
        DeviceGuard dg(B->device);
        batch_clear_graphs(B);
        B->max_group = max_boxes;
    }
    return FSEI_OK;
}

int32_t fsei_batch_launch_groups(fsei_batch B) { return B ? B->ngroups : 0; }

fsei_status fsei_batch_autotune(fsei_batch B, int32_t flags, void *cuda_stream) {
    NvtxRange nvtx_call("fsei_batch_autotune");
    g_err.clear();
    if (!B) return fail(FSEI_E_ARG, "fsei_batch_autotune: NULL batch");
    DeviceGuard dg(B->device);
    cudaDeviceSynchronize();
    batch_clear_graphs(B);
    // one measurement per shape: later boxes of a tuned shape take the
    // cached schedule (FSEI_TUNE_FORCE applies to the first box of a shape)
    std::vector<ScheduleKey> done;
    for (size_t i = 0; i < B->grids.size(); ++i) {
        const ScheduleKey k = schedule_key(B->grids[i]);
        bool seen = false;
        for (const ScheduleKey &d : done) seen = seen || d == k;
        const fsei_status r = fsei_grid_autotune(B->grids[i], seen ? 0 : flags, cuda_stream, nullptr);
        if (r != FSEI_OK) {
            const std::string msg = g_err;
            return fail(r, "box %zu: %s", i, msg.c_str());
        }
        done.push_back(k);
    }
    // then each shape with two or more boxes, timed as its grouped launches
    std::vector<ScheduleKey> keys;
    for (size_t i = 0; i < B->grids.size(); ++i) {
        const ScheduleKey k = schedule_key(B->grids[i]);
        if (std::find(keys.begin(), keys.end(), k) != keys.end()) continue;
        keys.push_back(k);
        std::vector<size_t> idx;
        for (size_t j = i; j < B->grids.size(); ++j)
            if (schedule_key(B->grids[j]) == k && B->desc_key[j] == B->desc_key[i]) idx.push_back(j);
        if (idx.size() < 2) continue;
        const fsei_status r =
            tune_group(B, idx, (cudaStream_t)cuda_stream, (flags & FSEI_TUNE_FORCE) != 0);
        if (r != FSEI_OK) return r;
    }
    batch_clear_graphs(B);
    return FSEI_OK;
}

// bounds-checking mode: the first box whose workspace guards changed
static fsei_status batch_guards(const fsei_batch_s *B, fsei_status st) {
    for (size_t i = 0; i < B->grids.size(); ++i) {
        const fsei_status g = guard_status(B->grids[i], "fsei_batch_step");
        if (g != FSEI_OK) return fail(g, "box %zu: %s", i, std::string(g_err).c_str());
    }
    return st;
}

fsei_status fsei_batch_step(fsei_batch B, fsei_state *states, const void *const *forces,
                            const fsei_step_params *prm, int32_t nsteps, void *cuda_stream,
                            fsei_step_stats *out) {
    NvtxRange nvtx_call("fsei_batch_step");
    g_err.clear();
    cudaGetLastError();   // an error left by an unrelated earlier call is not ours
    if (!B || !states || !prm) return fail(FSEI_E_ARG, "fsei_batch_step: NULL argument");
    if (nsteps < 0) return fail(FSEI_E_ARG, "nsteps < 0");
    const size_t nb = B->grids.size();
    for (size_t i = 0; i < nb; ++i) {
        const fsei_state &s = states[i];
        const void *req[7] = {s.u, s.v, s.w, s.p, s.hu, s.hv, s.hw};
        for (int c = 0; c < 7; ++c)
            if (!req[c] || !aligned16(req[c])) return fail(FSEI_E_ARG, "box %zu: state field %d NULL or misaligned", i, c);
        for (int c = 0; c < 3 && forces; ++c)
            if (forces[3 * i + c] && !aligned16(forces[3 * i + c])) return fail(FSEI_E_ARG, "box %zu: force %d misaligned", i, c);
        if (!(prm[i].re > 0)) return fail(FSEI_E_ARG, "box %zu: re must be > 0", i);
        if (!(prm[i].cfl > 0) && !(prm[i].dt > 0)) return fail(FSEI_E_ARG, "box %zu: need dt > 0 or cfl > 0", i);
        if (prm[i].scheme != FSEI_AB2_CN && prm[i].scheme != FSEI_RK3_CN)
            return fail(FSEI_E_ARG, "box %zu: unknown scheme %d", i, prm[i].scheme);
        if (check_rheology(prm[i], "fsei_batch_step") != FSEI_OK) {
            const std::string msg = g_err;
            return fail(prm[i].rheology == FSEI_CARREAU_YASUDA && prm[i].scheme != FSEI_AB2_CN
                            ? FSEI_E_UNSUPPORTED : FSEI_E_ARG, "box %zu: %s", i, msg.c_str());
        }
    }
    DeviceGuard dg(B->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (nsteps > 0) {
        // the captured graphs bake in pointers, forces, parameters and the
        // history flags: compare their bytes with the last capture
        std::vector<unsigned char> key;
        auto put = [&](const void *p, size_t n) {
            const unsigned char *c = static_cast<const unsigned char *>(p);
            key.insert(key.end(), c, c + n);
        };
        for (size_t i = 0; i < nb; ++i) {
            put(&states[i], sizeof(fsei_state));
            put(&prm[i], sizeof(fsei_step_params));
            for (int c = 0; c < 3; ++c) {
                const void *f = forces ? forces[3 * i + c] : nullptr;
                put(&f, sizeof f);
            }
        }
        if (key != B->key || !B->first) {
            batch_clear_graphs(B);
            fsei_status r = batch_capture(B, states, forces, prm, true, &B->first);
            if (r == FSEI_OK) r = batch_capture(B, states, forces, prm, false, &B->rest);
            if (r != FSEI_OK) {
                batch_clear_graphs(B);
                return r;
            }
            B->key = key;
        }
        if (cudaGraphLaunch(B->first, st) != cudaSuccess) return fail(FSEI_E_CUDA, "batch: graph launch failed");
        for (int n = 1; n < nsteps; ++n)
            if (cudaGraphLaunch(B->rest, st) != cudaSuccess) return fail(FSEI_E_CUDA, "batch: graph launch failed");
        // the history flags become 1; a following call therefore differs from
        // this capture (its key holds the flags) and is captured once more
        for (size_t i = 0; i < nb; ++i) states[i].have_prev_h = 1;
    }
    if (out) {
        for (size_t i = 0; i < nb; ++i)
            cudaMemcpyAsync(B->grids[i]->sc_host, B->grids[i]->sc, sizeof(StepScalars),
                            cudaMemcpyDeviceToHost, st);
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(FSEI_E_CUDA, "fsei_batch_step: %s", cudaGetErrorString(e));
        fsei_status worst = FSEI_OK;
        for (size_t i = 0; i < nb; ++i) {
            const StepScalars &h = *B->grids[i]->sc_host;
            out[i].dt_used = h.dt_step;
            out[i].cfl = h.dt_step * __builtin_bit_cast(double, h.speed_next);
            out[i].max_div = __builtin_bit_cast(double, h.maxdiv);
            out[i].kinetic_energy = h.ke;
            out[i].flags = h.flags;
            if (out[i].cfl > 1.0) out[i].flags |= FSEI_FLAG_CFL;
            if ((out[i].flags & FSEI_FLAG_NONFINITE) && worst == FSEI_OK) worst = fail(FSEI_E_NONFINITE, "box %zu: non-finite state", i);
            else if ((out[i].flags & FSEI_FLAG_CFL) && worst == FSEI_OK) worst = fail(FSEI_E_CFL, "box %zu: CFL %g above 1", i, out[i].cfl);
        }
        return batch_guards(B, worst);
    }
    return batch_guards(B, FSEI_OK);
}

}  // extern "C"
