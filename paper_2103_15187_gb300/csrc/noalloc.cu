// Allocation-free variant of the pressure Poisson solve.
//
// fsei_poisson_solve needs a grid handle, and fsei_grid_create allocates the
// handle's workspace with cudaMalloc.  Some callers cannot allocate device
// memory at the point where they need a solve: code running under a memory
// budget that is already fully reserved by a framework's caching allocator,
// plug-ins handed only raw device pointers by a host application that owns
// all allocation, or paths that must not add allocation calls (and the
// implicit synchronisation cudaMalloc/cudaFree bring) to a tight loop.
// fsei_poisson_solve_noalloc serves them: all of its scratch (mesh metrics,
// FFT twiddles, wavenumber tables and the spectrum) lives in one file-scope
// __device__ array of fixed size, so the call itself allocates nothing --
// neither device memory nor host heap memory (host tables are staged in a
// static host buffer).
//
// The array is part of the module: every GPU that loads the library holds
// it until the process exits.  All calls share it and it keeps the contents
// of the last call; the solve clears the part that must start at zero (the
// spectrum, whose row padding is never written by the transforms) on every
// call.  Calls whose work overlaps on the GPU (different streams, or
// different host threads) race on the array and must be serialised by the
// caller.
#include <math.h>
#include <string.h>

#include <mutex>

#include "../../include/fsei.h"
#include "kernels.cuh"

using namespace fsei;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FSEI_NOALLOC_SCRATCH_BYTES];

constexpr size_t kHostStageBytes = 4u << 20;   // host staging of the tables
constexpr int kMaxDevices = 64;

std::mutex g_noalloc_mutex;
unsigned char g_host_stage[kHostStageBytes];
unsigned char *g_dev_scratch[kMaxDevices] = {nullptr};

bool is_2a3b(int n) {
    if (n < 1) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// modified wavenumber (2 - 2 cos(2 pi k / n)) / h^2 in extended precision
__host__ double modified_wavenumber(int k, int n, double h) {
    const long double pi = 3.141592653589793238462643383279502884L;
    return (double)((2.0L - 2.0L * cosl(2.0L * pi * k / n)) / ((long double)h * h));
}

// exp(-2 pi i m / n) in extended precision
__host__ void unit_root(int m, int n, double *re, double *im) {
    const long double pi = 3.141592653589793238462643383279502884L;
    const long double ang = 2.0L * pi * (long double)m / (long double)n;
    *re = (double)cosl(ang);
    *im = (double)(-sinl(ang));
}

// Byte offsets of the regions inside the scratch array.
struct Layout {
    size_t sc, dz, idz, ihc, dzf, idzf, ihcf, twx, twy, twpost, lamx, lamy, lamxd, lamyd,
        exact, nzm, tables_end, spec, total;
};

template <typename T>
Layout layout_for(int nx, int ny, int nz, int sk, int nmodes) {
    const int mx = nx / 2;
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = align256(o + bytes); return at; };
    L.sc = take(sizeof(StepScalars));
    L.dz = take(sizeof(double) * nz);
    L.idz = take(sizeof(double) * nz);
    L.ihc = take(sizeof(double) * (nz + 1));
    L.dzf = take(sizeof(float) * nz);
    L.idzf = take(sizeof(float) * nz);
    L.ihcf = take(sizeof(float) * (nz + 1));
    L.twx = take(sizeof(cplx<T>) * mx);
    L.twy = take(sizeof(cplx<T>) * ny);
    L.twpost = take(sizeof(cplx<T>) * (mx + 1));
    L.lamx = take(sizeof(T) * sk);
    L.lamy = take(sizeof(T) * ny);
    L.lamxd = take(sizeof(double) * sk);
    L.lamyd = take(sizeof(double) * ny);
    L.exact = take((size_t)sk * ny);
    L.nzm = take(sizeof(int) * nmodes);
    L.tables_end = o;
    L.spec = take(sizeof(cplx<T>) * (size_t)sk * ny * nz);
    L.total = o;
    return L;
}

template <typename T>
fsei_status solve_noalloc(const fsei_grid_desc *d, const void *rhs, void *phi, cudaStream_t st,
                          unsigned char *dev) {
    const int nx = d->nx, ny = d->ny, nz = d->nz;
    const int mx = nx / 2;
    const int sk = ((mx + 1 + 15) / 16) * 16;
    const double dx = d->lx / nx, dy = d->ly / ny;

    // z faces and metrics (walls: tanh clustering on [-1, 1]; periodic: uniform)
    // staged directly in the host buffer
    unsigned char *H = g_host_stage;
    // count the exactly solved modes first (they size the layout)
    double lz;
    {
        if (d->zbc == FSEI_Z_PERIODIC) lz = d->lz;
        else if (d->zfaces) lz = d->zfaces[nz] - d->zfaces[0];
        else lz = 2.0;
    }
    auto lamx_of = [&](int kx) { return modified_wavenumber(kx, nx, dx); };
    auto lamy_of = [&](int ky) { return modified_wavenumber(ky, ny, dy); };
    const double tau = d->near_zero_tau > 0 ? d->near_zero_tau : 64.0;
    int nmodes = 1;
    if (d->prec == FSEI_MIXED)
        for (int ky = 0; ky < ny; ++ky)
            for (int kx = 0; kx <= mx; ++kx)
                if (!(kx == 0 && ky == 0) && (lamx_of(kx) + lamy_of(ky)) * lz * lz < tau) ++nmodes;

    const Layout L = layout_for<T>(nx, ny, nz, sk, nmodes);
    if (L.total > FSEI_NOALLOC_SCRATCH_BYTES || L.tables_end > kHostStageBytes)
        return FSEI_E_SHAPE;

    memset(H, 0, L.tables_end);
    double *hdz = (double *)(H + L.dz), *hidz = (double *)(H + L.idz), *hihc = (double *)(H + L.ihc);
    float *hdzf = (float *)(H + L.dzf), *hidzf = (float *)(H + L.idzf), *hihcf = (float *)(H + L.ihcf);
    // faces: computed on the fly into dz via two-point differences
    auto face = [&](int k) -> double {
        if (d->zbc == FSEI_Z_PERIODIC) return k * (d->lz / nz);
        if (d->zfaces) return d->zfaces[k];
        if (d->stretch > 0) return tanh(d->stretch * (2.0 * k / nz - 1.0)) / tanh(d->stretch);
        return -1.0 + 2.0 * k / nz;
    };
    for (int k = 0; k < nz; ++k) {
        hdz[k] = face(k + 1) - face(k);
        if (!(hdz[k] > 0)) return FSEI_E_ARG;
    }
    double hc0 = 0, hcn = 0;
    if (d->zbc == FSEI_Z_WALLS) {
        hc0 = 0.5 * hdz[0];
        hcn = 0.5 * hdz[nz - 1];
    } else {
        hc0 = hcn = 0.5 * (hdz[nz - 1] + hdz[0]);
    }
    for (int k = 0; k <= nz; ++k) {
        double hc;
        if (k == 0) hc = hc0;
        else if (k == nz) hc = hcn;
        else hc = 0.5 * (face(k + 1) + face(k)) - 0.5 * (face(k) + face(k - 1));
        hihc[k] = 1.0 / hc;
        hihcf[k] = (float)hihc[k];
    }
    for (int k = 0; k < nz; ++k) {
        hidz[k] = 1.0 / hdz[k];
        hdzf[k] = (float)hdz[k];
        hidzf[k] = (float)hidz[k];
    }
    auto tw = [&](int n, int count, cplx<T> *out) {
        for (int m = 0; m < count; ++m) {
            double re, im;
            unit_root(m, n, &re, &im);
            out[m] = cplx<T>{T(re), T(im)};
        }
    };
    tw(mx, mx, (cplx<T> *)(H + L.twx));
    tw(ny, ny, (cplx<T> *)(H + L.twy));
    tw(nx, mx + 1, (cplx<T> *)(H + L.twpost));
    T *hlx = (T *)(H + L.lamx), *hly = (T *)(H + L.lamy);
    double *hlxd = (double *)(H + L.lamxd), *hlyd = (double *)(H + L.lamyd);
    for (int kx = 0; kx < sk; ++kx) { hlxd[kx] = lamx_of(kx); hlx[kx] = T(hlxd[kx]); }
    for (int ky = 0; ky < ny; ++ky) { hlyd[ky] = lamy_of(ky); hly[ky] = T(hlyd[ky]); }
    unsigned char *hex = H + L.exact;
    int *hm = (int *)(H + L.nzm);
    int nm = 0;
    hm[nm++] = 0;
    hex[0] = 1;
    if (d->prec == FSEI_MIXED)
        for (int ky = 0; ky < ny; ++ky)
            for (int kx = 0; kx <= mx; ++kx)
                if (!(kx == 0 && ky == 0) && (hlxd[kx] + hlyd[ky]) * lz * lz < tau) {
                    hm[nm++] = kx + sk * ky;
                    hex[kx + (size_t)sk * ky] = 1;
                }

    // device views
    GridDev g;
    memset(&g, 0, sizeof g);
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.walls = d->zbc == FSEI_Z_WALLS;
    g.mx = mx; g.sk = sk;
    g.dx = dx; g.dy = dy;
    g.idx = 1.0 / dx; g.idy = 1.0 / dy;
    g.idx2 = g.idx * g.idx; g.idy2 = g.idy * g.idy;
    grid_float_copies(g);
    g.dz = (const double *)(dev + L.dz);
    g.idz = (const double *)(dev + L.idz);
    g.ihc = (const double *)(dev + L.ihc);
    g.dzf = (const float *)(dev + L.dzf);
    g.idzf = (const float *)(dev + L.idzf);
    g.ihcf = (const float *)(dev + L.ihcf);
    Work<T> W;
    memset(&W, 0, sizeof W);
    W.spec = (cplx<T> *)(dev + L.spec);
    W.twx = (const cplx<T> *)(dev + L.twx);
    W.twy = (const cplx<T> *)(dev + L.twy);
    W.twpost = (const cplx<T> *)(dev + L.twpost);
    W.lamx = (const T *)(dev + L.lamx);
    W.lamy = (const T *)(dev + L.lamy);
    W.lamx_d = (const double *)(dev + L.lamxd);
    W.lamy_d = (const double *)(dev + L.lamyd);
    W.exact = (const unsigned char *)(dev + L.exact);
    W.nzm = (const int *)(dev + L.nzm);
    W.n_nzm = nm;
    // launch geometry (same rules as a grid handle of this shape)
    const int tsz = (int)sizeof(T);
    W.ry = 1;
    for (int r = (tsz == 8 ? 4 : 8); r >= 1; r /= 2)
        if (ny % r == 0) { W.ry = r; break; }
    poisson_geometry<T>(g, W);
    W.fpx.n = mx;
    W.fpy.n = ny;
    for (FftPlanDev *fp : {&W.fpx, &W.fpy}) {
        int m = fp->n;
        fp->nr = 0;
        while (m % 4 == 0) { fp->rad[fp->nr++] = 4; m /= 4; }
        while (m % 2 == 0) { fp->rad[fp->nr++] = 2; m /= 2; }
        while (m % 3 == 0) { fp->rad[fp->nr++] = 3; m /= 3; }
    }

    // upload the tables (one copy from the static host stage), clear the
    // spectrum, run the transform / z-solve chain
    if (cudaMemcpyAsync(dev, H, L.tables_end, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FSEI_E_CUDA;
    if (cudaMemsetAsync(W.spec, 0, sizeof(cplx<T>) * (size_t)sk * ny * nz, st) != cudaSuccess)
        return FSEI_E_CUDA;
    StepScalars *sc = (StepScalars *)(dev + L.sc);
    launch_rfft_x<T>(g, W, sc, (const T *)rhs, 1, st);
    launch_fft_y<T>(g, W, 0, st);
    launch_poisson_z<T>(g, W, st);
    launch_fft_y<T>(g, W, 1, st);
    launch_irfft_x<T>(g, W, (T *)phi, st);
    // the host stage may be reused by the next call only after the copy
    // above has consumed it; a pageable-memory copy has by the time it
    // returns, so no further wait is needed here
    return cudaGetLastError() == cudaSuccess ? FSEI_OK : FSEI_E_CUDA;
}

}  // namespace

extern "C" fsei_status fsei_poisson_solve_noalloc(const fsei_grid_desc *d, const void *rhs,
                                                  void *phi, void *cuda_stream) {
    if (!d || !rhs || !phi) return FSEI_E_ARG;
    if ((((uintptr_t)rhs) & 15u) || (((uintptr_t)phi) & 15u)) return FSEI_E_ARG;
    const int nx = d->nx, ny = d->ny, nz = d->nz;
    if (nx < 8 || nx % 2 || !is_2a3b(nx / 2) || nx / 2 > 1024) return FSEI_E_SHAPE;
    if (ny < 4 || ny % 2 || !is_2a3b(ny) || ny > 1024) return FSEI_E_SHAPE;
    if (nz < 8 || nz > 2048) return FSEI_E_SHAPE;
    if (!(d->lx > 0) || !(d->ly > 0)) return FSEI_E_ARG;
    if (d->zbc != FSEI_Z_PERIODIC && d->zbc != FSEI_Z_WALLS) return FSEI_E_ARG;
    if (d->prec != FSEI_FP64 && d->prec != FSEI_MIXED) return FSEI_E_ARG;
    if (d->zbc == FSEI_Z_PERIODIC && (!(d->lz > 0) || d->zfaces)) return FSEI_E_ARG;
    if (!(d->stretch >= 0)) return FSEI_E_ARG;
    // a captured call would record copies from the static host buffer,
    // which later calls overwrite: capture is refused
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing((cudaStream_t)cuda_stream, &cs) != cudaSuccess) return FSEI_E_CUDA;
        if (cs != cudaStreamCaptureStatusNone) return FSEI_E_ARG;
    }

    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FSEI_E_CUDA;
    if (!g_dev_scratch[dev]) {
        // once per device, with that device current: the device address of
        // the file-scope array (its host-side name is only a stand-in)
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FSEI_E_CUDA;
        g_dev_scratch[dev] = static_cast<unsigned char *>(p);
        // the transform and z-solve kernels' shared-memory limits, also once
        // per device (the attributes are per device and process-wide)
        GridDev g0;
        memset(&g0, 0, sizeof g0);
        Work<double> wd;
        memset(&wd, 0, sizeof wd);
        Work<float> wf;
        memset(&wf, 0, sizeof wf);
        set_smem_limits_poisson<double>(g0, wd);
        set_smem_limits_poisson<float>(g0, wf);
        if (cudaGetLastError() != cudaSuccess) {
            g_dev_scratch[dev] = nullptr;
            return FSEI_E_CUDA;
        }
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaGetLastError();   // an error left by an unrelated earlier call is not ours
    return d->prec == FSEI_FP64
               ? solve_noalloc<double>(d, rhs, phi, st, g_dev_scratch[dev])
               : solve_noalloc<float>(d, rhs, phi, st, g_dev_scratch[dev]);
}
