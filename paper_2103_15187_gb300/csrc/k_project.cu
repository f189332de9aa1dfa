// Projection and pressure update of the fractional step (Sec. 2.1): with the
// pressure increment phi from the Poisson solve,
//     u^{n+1} = u* - dt G phi,   p^{n+1} = p^n + phi - beta (D G) phi,
// beta = dt / (2 Re).  Fused reductions of the new state: max |D u^{n+1}|,
// kinetic energy, and max |u_c|/dx + |v_c|/dy + |w_c|/dz_k (the CFL speed
// that sets the next step's dt).  Per-cell statistics are evaluated in the
// field precision and reduced within each warp in it; the block and
// grid-wide accumulation is in double.
#include "kernels.cuh"

namespace fsei {

namespace {

// One block per (j, k) row group: blockIdx.x = k * (ny / rows) + row tile,
// threads stride over x.  No integer division per element.
template <typename T>
FSEI_D void
k_project(GridDev g, Fields<T> F, const T *__restrict__ q0, const T *__restrict__ q1,
          const T *__restrict__ q2, const T *__restrict__ phi, StepScalars *sc, int rows) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int nbj = ny / rows;
    const int k = blockIdx.x / nbj, j0 = (blockIdx.x % nbj) * rows;
    const T dt = fpick<T>(sc->dt, sc->fdt), beta = fpick<T>(sc->beta, sc->fbeta);
    const T idx = fpick<T>(g.idx, g.fidx), idy = fpick<T>(g.idy, g.fidy);
    const T idx2 = fpick<T>(g.idx2, g.fidx2), idy2 = fpick<T>(g.idy2, g.fidy2);
    const T *idz = Metric<T>::idz(g), *ihc = Metric<T>::ihc(g);
    const bool hasdn = !g.walls || k > 0, hasup = !g.walls || k < nz - 1;
    const int kd = k == 0 ? nz - 1 : k - 1, ku = k == nz - 1 ? 0 : k + 1;
    const T ihck = ihc[k], ihcu = ihc[k + 1], idzk = idz[k];
    const T vxy = fpick<T>(g.dx * g.dy, g.fvxy);
    const T vu = vxy * Metric<T>::dz(g)[k];
    const T vw = hasdn ? vxy / ihck : T(0);
    T mdiv = T(0), mspd = T(0), kel = T(0);
    int flags = 0;
#pragma unroll 2
    for (int r = 0; r < rows; ++r) {
        const int j = j0 + r;
        const int jp = j == ny - 1 ? 0 : j + 1, jm = j == 0 ? ny - 1 : j - 1;
        // 32-bit row offsets once per row (no wide multiplies in the x loop)
        const int oc = (k * ny + j) * nx, ojm = (k * ny + jm) * nx, ojp = (k * ny + jp) * nx,
                  okd = (kd * ny + j) * nx, oku = (ku * ny + j) * nx;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const int ip = i == nx - 1 ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
            const int c = oc + i;
            const T f0 = phi[c];
            const T fim = phi[oc + im], fip = phi[oc + ip];
            const T fjm = phi[ojm + i], fjp = phi[ojp + i];
            const T fkd = hasdn ? phi[okd + i] : T(0);
            const T fku = hasup ? phi[oku + i] : T(0);
            const T un = q0[c] - dt * (f0 - fim) * idx;
            const T vn = q1[c] - dt * (f0 - fjm) * idy;
            const T wn = hasdn ? q2[c] - dt * (f0 - fkd) * ihck : T(0);
            const T fup = hasup ? (fku - f0) * ihcu : T(0);
            const T fdn = hasdn ? (f0 - fkd) * ihck : T(0);
            const T lphi = (fip - T(2) * f0 + fim) * idx2 + (fjp - T(2) * f0 + fjm) * idy2 +
                           (fup - fdn) * idzk;
            const T pn = F.p[c] + f0 - beta * lphi;
            F.u[c] = un;
            F.v[c] = vn;
            F.w[c] = wn;
            F.p[c] = pn;
            // neighbours of the new state needed by the cell-centre statistics
            const T uip = q0[oc + ip] - dt * (fip - f0) * idx;
            const T vjp = q1[ojp + i] - dt * (fjp - f0) * idy;
            const T wku = hasup ? q2[oku + i] - dt * (fku - f0) * ihcu : T(0);
            const T di = (uip - un) * idx + (vjp - vn) * idy + (wku - wn) * idzk;
            mdiv = fmax(mdiv, fabs(di));
            const T sp = fabs(T(0.5) * (un + uip)) * idx + fabs(T(0.5) * (vn + vjp)) * idy +
                         fabs(T(0.5) * (wn + wku)) * idzk;
            mspd = fmax(mspd, sp);
            kel += T(0.5) * ((un * un + vn * vn) * vu + wn * wn * vw);
            if (!isfinite(un) || !isfinite(vn) || !isfinite(wn) || !isfinite(pn)) flags |= 1;
        }
    }
    // warp level in the field precision (the maxima are exact in it; the
    // energy partials are sums of at most a few hundred cells), block and
    // grid level in double
    for (int o = 16; o > 0; o >>= 1) {
        mdiv = fmax(mdiv, __shfl_down_sync(0xffffffffu, mdiv, o));
        mspd = fmax(mspd, __shfl_down_sync(0xffffffffu, mspd, o));
        kel += __shfl_down_sync(0xffffffffu, kel, o);
        flags |= __shfl_down_sync(0xffffffffu, flags, o);
    }
    __shared__ double sdiv[32], sspd[32], ske[32];
    __shared__ int sfl[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sdiv[wid] = (double)mdiv;
        sspd[wid] = (double)mspd;
        ske[wid] = (double)kel;
        sfl[wid] = flags;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        double dd = 0.0, ds = 0.0, ke = 0.0;
        int fl = 0;
        for (int w = 0; w < nw; ++w) {
            dd = fmax(dd, sdiv[w]);
            ds = fmax(ds, sspd[w]);
            ke += ske[w];
            fl |= sfl[w];
        }
        atomicMax(&sc->maxdiv, dbits(dd));
        atomicMax(&sc->speed_next, dbits(ds));
        atomicAdd(&sc->ke, ke);
        if (fl) atomicOr(&sc->flags, fl);
    }
}

// Same computation with 16-byte vector accesses: a thread owns W = 16 /
// sizeof(T) consecutive cells of a row (4 in single, 2 in double
// precision), loads every centre and y/z-neighbour vector of its rows
// before using them, and takes the x neighbours outside its vector (i0 - 1,
// i0 + W, periodic) as scalars.  Needs nx % W == 0 (16-byte aligned rows).
// A block covers `rows` rows of plane k; tpr = nx / W threads span a row,
// rpp = blockDim / tpr rows run side by side (one if a row needs more).
// The per-cell arithmetic and its order are those of k_project.
template <typename T> struct alignas(16) Vec16 {
    static constexpr int W = 16 / (int)sizeof(T);
    T v[W];
};

template <typename T>
FSEI_D void
k_project_vec(GridDev g, Fields<T> F, const T *__restrict__ q0, const T *__restrict__ q1,
              const T *__restrict__ q2, const T *__restrict__ phi, StepScalars *sc, int rows) {
    pdl_wait();
    pdl_trigger();
    using V = Vec16<T>;
    constexpr int W = V::W;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int tpr = nx / W;
    const int nthr = (int)blockDim.x;
    const int rpp = tpr >= nthr ? 1 : nthr / tpr;
    const int xt = tpr >= nthr ? (int)threadIdx.x : (int)threadIdx.x % tpr;
    const int r0 = tpr >= nthr ? 0 : (int)threadIdx.x / tpr;
    const int xstride = tpr >= nthr ? nthr : tpr;
    const int nbj = ny / rows;
    const int k = blockIdx.x / nbj, j0 = (blockIdx.x % nbj) * rows;
    const T dt = fpick<T>(sc->dt, sc->fdt), beta = fpick<T>(sc->beta, sc->fbeta);
    const T idx = fpick<T>(g.idx, g.fidx), idy = fpick<T>(g.idy, g.fidy);
    const T idx2 = fpick<T>(g.idx2, g.fidx2), idy2 = fpick<T>(g.idy2, g.fidy2);
    const T *idz = Metric<T>::idz(g), *ihc = Metric<T>::ihc(g);
    const bool hasdn = !g.walls || k > 0, hasup = !g.walls || k < nz - 1;
    const int kd = k == 0 ? nz - 1 : k - 1, ku = k == nz - 1 ? 0 : k + 1;
    const T ihck = ihc[k], ihcu = ihc[k + 1], idzk = idz[k];
    const T vxy = fpick<T>(g.dx * g.dy, g.fvxy);
    const T vu = vxy * Metric<T>::dz(g)[k];
    const T vw = hasdn ? vxy / ihck : T(0);
    T mdiv = T(0), mspd = T(0), kel = T(0);
    int flags = 0;
    const bool on = r0 < rpp && r0 < rows;
    for (int r = r0; on && r < rows; r += rpp) {
        const int j = j0 + r;
        const int jp = j == ny - 1 ? 0 : j + 1, jm = j == 0 ? ny - 1 : j - 1;
        const int oc = (k * ny + j) * nx, ojm = (k * ny + jm) * nx, ojp = (k * ny + jp) * nx,
                  okd = (kd * ny + j) * nx, oku = (ku * ny + j) * nx;
        for (int xv = xt; xv < tpr; xv += xstride) {
            const int i0 = xv * W;
            const int il = i0 == 0 ? nx - 1 : i0 - 1, ir = i0 + W == nx ? 0 : i0 + W;
            const int c = oc + i0;
            const V f0 = *reinterpret_cast<const V *>(phi + c);
            const V fjm = *reinterpret_cast<const V *>(phi + ojm + i0);
            const V fjp = *reinterpret_cast<const V *>(phi + ojp + i0);
            V fkd, fku, a2u;
            if (hasdn) fkd = *reinterpret_cast<const V *>(phi + okd + i0);
            if (hasup) {
                fku = *reinterpret_cast<const V *>(phi + oku + i0);
                a2u = *reinterpret_cast<const V *>(q2 + oku + i0);
            }
            const V a0 = *reinterpret_cast<const V *>(q0 + c);
            const V a1 = *reinterpret_cast<const V *>(q1 + c);
            const V a1p = *reinterpret_cast<const V *>(q1 + ojp + i0);
            const V a2 = *reinterpret_cast<const V *>(q2 + c);
            const V pc = *reinterpret_cast<const V *>(F.p + c);
            const T fl = phi[oc + il], fr = phi[oc + ir], a0r = q0[oc + ir];
            V un, vn, wn, pn;
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const T ff = f0.v[e];
                const T fim = e == 0 ? fl : f0.v[e - 1];
                const T fip = e == W - 1 ? fr : f0.v[e + 1];
                const T fkde = hasdn ? fkd.v[e] : T(0);
                const T fkue = hasup ? fku.v[e] : T(0);
                const T u1 = a0.v[e] - dt * (ff - fim) * idx;
                const T v1 = a1.v[e] - dt * (ff - fjm.v[e]) * idy;
                const T w1 = hasdn ? a2.v[e] - dt * (ff - fkde) * ihck : T(0);
                const T fup = hasup ? (fkue - ff) * ihcu : T(0);
                const T fdn = hasdn ? (ff - fkde) * ihck : T(0);
                const T lphi = (fip - T(2) * ff + fim) * idx2 +
                               (fjp.v[e] - T(2) * ff + fjm.v[e]) * idy2 + (fup - fdn) * idzk;
                const T p1 = pc.v[e] + ff - beta * lphi;
                un.v[e] = u1;
                vn.v[e] = v1;
                wn.v[e] = w1;
                pn.v[e] = p1;
                const T a0n = e == W - 1 ? a0r : a0.v[e + 1];
                const T uip = a0n - dt * (fip - ff) * idx;
                const T vjp = a1p.v[e] - dt * (fjp.v[e] - ff) * idy;
                const T wku = hasup ? a2u.v[e] - dt * (fkue - ff) * ihcu : T(0);
                const T di = (uip - u1) * idx + (vjp - v1) * idy + (wku - w1) * idzk;
                mdiv = fmax(mdiv, fabs(di));
                const T sp = fabs(T(0.5) * (u1 + uip)) * idx + fabs(T(0.5) * (v1 + vjp)) * idy +
                             fabs(T(0.5) * (w1 + wku)) * idzk;
                mspd = fmax(mspd, sp);
                kel += T(0.5) * ((u1 * u1 + v1 * v1) * vu + w1 * w1 * vw);
                if (!isfinite(u1) || !isfinite(v1) || !isfinite(w1) || !isfinite(p1)) flags |= 1;
            }
            *reinterpret_cast<V *>(F.u + c) = un;
            *reinterpret_cast<V *>(F.v + c) = vn;
            *reinterpret_cast<V *>(F.w + c) = wn;
            *reinterpret_cast<V *>(F.p + c) = pn;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mdiv = fmax(mdiv, __shfl_down_sync(0xffffffffu, mdiv, o));
        mspd = fmax(mspd, __shfl_down_sync(0xffffffffu, mspd, o));
        kel += __shfl_down_sync(0xffffffffu, kel, o);
        flags |= __shfl_down_sync(0xffffffffu, flags, o);
    }
    __shared__ double sdiv[32], sspd[32], ske[32];
    __shared__ int sfl[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sdiv[wid] = (double)mdiv;
        sspd[wid] = (double)mspd;
        ske[wid] = (double)kel;
        sfl[wid] = flags;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        double dd = 0.0, ds = 0.0, ke = 0.0;
        int fl = 0;
        for (int w = 0; w < nw; ++w) {
            dd = fmax(dd, sdiv[w]);
            ds = fmax(ds, sspd[w]);
            ke += ske[w];
            fl |= sfl[w];
        }
        atomicMax(&sc->maxdiv, dbits(dd));
        atomicMax(&sc->speed_next, dbits(ds));
        atomicAdd(&sc->ke, ke);
        if (fl) atomicOr(&sc->flags, fl);
    }
}

// the kernels with their launch bounds
template <typename T> constexpr Kernel<k_project<T>, 256, 0> K_project{};
template <typename T> constexpr Kernel<k_project_vec<T>, 256, 0> K_project_vec{};

}  // namespace

int project_rows(const GridDev &g) {
    for (int r = 8; r >= 1; r /= 2)
        if (g.ny % r == 0) return r;
    return 1;
}

template <typename T> void launch_project(const GridDev &g, const Fields<T> &F, Work<T> &W,
                                          StepScalars *sc, cudaStream_t st) {
    constexpr int VW = 16 / (int)sizeof(T);
    if (g.nx % VW == 0) {
        // vector path: 128 threads, rows side by side, about four passes per
        // thread by default (the per-thread set-up and the block's reduction
        // are then spread over more cells; the grid's autotuner may pick
        // another count)
        const int tpr = g.nx / VW;
        const int rpp = tpr >= 128 ? 1 : 128 / tpr;
        const int mult = W.proj_mult > 0 ? W.proj_mult : 4;
        int rows = 1;
        for (int r = mult * rpp; r >= 1; --r)
            if (g.ny % r == 0) { rows = r; break; }
        K_project_vec<T>.launch(W.pdl != 0, dim3(g.nz * (g.ny / rows)), dim3(128), 0, st, g, F,
                                W.q0, W.q1, W.q2, W.phi, sc, rows);
        return;
    }
    const int rows = project_rows(g);
    const int threads = g.nx >= 256 ? 256 : ((g.nx + 31) / 32) * 32;
    K_project<T>.launch(false, dim3(g.nz * (g.ny / rows)), dim3(threads), 0, st, g, F, W.q0, W.q1,
                        W.q2, W.phi, sc, rows);
}

template <typename T> void preload_project() {
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, K_project<T>.solo());
    cudaFuncGetAttributes(&fa, K_project_vec<T>.solo());
}
template void preload_project<float>();
template void preload_project<double>();

template void launch_project<float>(const GridDev &, const Fields<float> &, Work<float> &,
                                    StepScalars *, cudaStream_t);
template void launch_project<double>(const GridDev &, const Fields<double> &, Work<double> &,
                                     StepScalars *, cudaStream_t);

}  // namespace fsei
