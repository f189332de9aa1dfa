// Discrete adjoint of one fractional step (Sec. 2.1, Eq. 3; Sec. 3.1): the
// exact transpose, in the Euclidean inner product of the stored arrays, of
//   (u^n, p^n, H^{n-1}, f) -> (u^{n+1}, p^{n+1}, H^n)
// at a frozen dt.  With V the cell volumes and W the z weights (dz_k at
// z-centre points, hc_k at z-faces) the linear pieces transpose as
//   G^T = -V D W_f^-1-form stencils written out below,
//   (I - beta L_z)^-T = W (I - beta L_z)^-1 W^-1,  L_z^T = W L_z W^-1,
//   (D G)^+T = V (D G)^+ V^-1 on compatible right-hand sides,
// x and y operators being symmetric.  Kernels, in call order:
//   k_adj_phibar   x = V^-1 phi-bar, phi-bar = -dt G^T u-bar + p-bar
//                  - beta (DG)^T p-bar          (then the Poisson chain)
//   k_adj_ustar    u*-bar = u-bar - (W_f / dt) G psi;  q = u*-bar / W
//   k_sweep_z<1>   q = W (I - beta L_z)^-1 q    (the forward z kernel)
//   k_sweep_y      q = (I - beta L_y)^-1 q
//   k_sweep_x      q = (I - beta L_x)^-1 q      (= RHS-bar)
//   k_adj_hist     Hb = dt gamma q + H-bar;  H-bar_out = dt rho q;
//                  f-bar += dt q
//   k_adj_gather   u-bar = u*-bar + dt/Re L^T q + J_A(u^n)^T Hb;
//                  p-bar -= dt G^T q
#include "kernels.cuh"
#include "rhs_row.cuh"
#include "tri.cuh"

namespace fsei {

namespace {

// neighbour access with periodic x, y and periodic or walled z (out-of-range
// z reads give 0 with walls)
struct Nb {
    int nx, ny, nz, walls;
    FSEI_D int wxi(int i) const { return i < 0 ? i + nx : (i >= nx ? i - nx : i); }
    FSEI_D int wyi(int j) const { return j < 0 ? j + ny : (j >= ny ? j - ny : j); }
    FSEI_D int wzi(int k) const { return k < 0 ? k + nz : (k >= nz ? k - nz : k); }
    FSEI_D bool zin(int k) const { return !walls || (k >= 0 && k < nz); }
    template <typename T> FSEI_D T at(const T *f, int i, int j, int k) const {
        if (!zin(k)) return T(0);
        return f[((size_t)wzi(k) * ny + wyi(j)) * nx + wxi(i)];
    }
};

FSEI_D size_t fid(int i, int j, int k, int nx, int ny) {
    return ((size_t)k * ny + j) * nx + i;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_adj_phibar(GridDev g, const T *__restrict__ ub, const T *__restrict__ vb,
             const T *__restrict__ wb, const T *__restrict__ pb, T *__restrict__ x,
             const StepScalars *sc) {
    const Nb N{g.nx, g.ny, g.nz, g.walls};
    const int j = blockIdx.x % g.ny, k = blockIdx.x / g.ny;
    const T dt = fpick<T>(sc->dt, sc->fdt), beta = fpick<T>(sc->beta, sc->fbeta);
    const T idx = fpick<T>(g.idx, g.fidx), idy = fpick<T>(g.idy, g.fidy);
    const T idx2 = fpick<T>(g.idx2, g.fidx2), idy2 = fpick<T>(g.idy2, g.fidy2);
    const T *idz = Metric<T>::idz(g), *ihc = Metric<T>::ihc(g), *dz = Metric<T>::dz(g);
    const int nz = g.nz;
    const bool walls = g.walls != 0;
    const int kd = N.wzi(k - 1), ku = N.wzi(k + 1);
    const T inv_vol = T(g.idx * g.idy) * idz[k];
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
        // G^T u-bar
        const T cz0 = (walls && k == 0) ? T(0) : N.at(wb, i, j, k) * ihc[k];
        const T cz1 = (walls && k == nz - 1) ? T(0) : N.at(wb, i, j, k + 1) * ihc[k + 1];
        const T gtu = (N.at(ub, i, j, k) - N.at(ub, i + 1, j, k)) * idx +
                      (N.at(vb, i, j, k) - N.at(vb, i, j + 1, k)) * idy + (cz0 - cz1);
        // (DG)^T p-bar = lap_xy(p-bar) + dz_k lapz((p-bar) / dz)
        const T p0 = N.at(pb, i, j, k);
        const T lxy = (N.at(pb, i + 1, j, k) - T(2) * p0 + N.at(pb, i - 1, j, k)) * idx2 +
                      (N.at(pb, i, j + 1, k) - T(2) * p0 + N.at(pb, i, j - 1, k)) * idy2;
        const T q0 = p0 * idz[k];
        const T fup = (walls && k == nz - 1) ? T(0) : (N.at(pb, i, j, k + 1) * idz[ku] - q0) * ihc[k + 1];
        const T fdn = (walls && k == 0) ? T(0) : (q0 - N.at(pb, i, j, k - 1) * idz[kd]) * ihc[k];
        const T lp = lxy + dz[k] * (fup - fdn) * idz[k];
        const T phib = -dt * gtu + p0 - beta * lp;
        x[fid(i, j, k, g.nx, g.ny)] = phib * inv_vol;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_adj_ustar(GridDev g, T *__restrict__ ub, T *__restrict__ vb, T *__restrict__ wb,
            const T *__restrict__ psi, T *__restrict__ q0, T *__restrict__ q1,
            T *__restrict__ q2, const StepScalars *sc) {
    const Nb N{g.nx, g.ny, g.nz, g.walls};
    const int j = blockIdx.x % g.ny, k = blockIdx.x / g.ny;
    const T idt = fpick<T>(sc->invdt, sc->finvdt);
    const T *dz = Metric<T>::dz(g), *idz = Metric<T>::idz(g), *ihc = Metric<T>::ihc(g);
    const T dxv = fpick<T>(g.dx, g.fdx), dyv = fpick<T>(g.dy, g.fdy);
    const bool wall_face = g.walls && k == 0;
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
        const size_t c = fid(i, j, k, g.nx, g.ny);
        const T s0 = psi[c];
        const T us = ub[c] - dyv * dz[k] * (s0 - N.at(psi, i - 1, j, k)) * idt;
        const T vs = vb[c] - dxv * dz[k] * (s0 - N.at(psi, i, j - 1, k)) * idt;
        const T ws = wall_face ? T(0) : wb[c] - dxv * dyv * (s0 - N.at(psi, i, j, k - 1)) * idt;
        ub[c] = us;
        vb[c] = vs;
        wb[c] = ws;
        q0[c] = us * idz[k];
        q1[c] = vs * idz[k];
        q2[c] = ws * ihc[k];
    }
}

// x sweep of the adjoint: q = (I - beta L_x)^-T q = (I - beta L_x)^-1 q (the
// uniform periodic matrix is symmetric).  A block owns ry rows of one
// component in plane k; thread t < ry P owns chunk t / ry of row t % ry.
template <typename T, int L>
__global__ void __launch_bounds__(256)
k_sweep_x(GridDev g, T *__restrict__ q0, T *__restrict__ q1, T *__restrict__ q2,
          const StepScalars *sc, int ry, int P) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sd = reinterpret_cast<T *>(smraw);
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int es = ry | 1;
    T *car = sd + (size_t)nx * es;
    const int nby = ny / ry;
    int b = blockIdx.x;
    const int jb = b % nby; b /= nby;
    const int k = b % nz;
    const int comp = b / nz;
    T *q = comp == 0 ? q0 : (comp == 1 ? q1 : q2);
    const int j0 = jb * ry;
    for (int e = threadIdx.x; e < ry * nx; e += blockDim.x) {
        const int r = e / nx, i = e - r * nx;
        sd[i * es + r] = q[fid(i, j0 + r, k, nx, ny)];
    }
    __syncthreads();
    {
        const int t = threadIdx.x;
        const bool active = t < ry * P;
        const int p = active ? t / ry : 0, l = active ? t - p * ry : 0;
        const int s0 = chunk_start(p, nx, P);
        const int len = active ? chunk_start(p + 1, nx, P) - s0 : 0;
        T d[L];
#pragma unroll
        for (int i = 0; i < L; ++i)
            if (i < len) d[i] = sd[(s0 + i) * es + l];
        uni_solve<T, L>(d, len, active, l, p, ry, nx, P, fpick<T>(sc->ax, sc->fax),
                        fpick<T>(sc->cix, sc->fcix), car);
#pragma unroll
        for (int i = 0; i < L; ++i)
            if (i < len) sd[(s0 + i) * es + l] = d[i];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ry * nx; e += blockDim.x) {
        const int r = e / nx, i = e - r * nx;
        q[fid(i, j0 + r, k, nx, ny)] = sd[i * es + r];
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_adj_hist(GridDev g, const T *__restrict__ q0, const T *__restrict__ q1,
           const T *__restrict__ q2, T *__restrict__ hbu, T *__restrict__ hbv,
           T *__restrict__ hbw, T *__restrict__ h0, T *__restrict__ h1, T *__restrict__ h2,
           T *fbx, T *fby, T *fbz, const StepScalars *sc) {
    const int j = blockIdx.x % g.ny, k = blockIdx.x / g.ny;
    const T dt = fpick<T>(sc->dt, sc->fdt), gam = fpick<T>(sc->gamma, sc->fgamma);
    const T rho = fpick<T>(sc->rho, sc->frho);
    const bool wall_face = g.walls && k == 0;
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
        const size_t c = fid(i, j, k, g.nx, g.ny);
        const T a = q0[c], b = q1[c], cc = wall_face ? T(0) : q2[c];
        h0[c] = dt * gam * a + hbu[c];
        h1[c] = dt * gam * b + hbv[c];
        h2[c] = wall_face ? T(0) : dt * gam * cc + hbw[c];
        hbu[c] = dt * rho * a;
        hbv[c] = dt * rho * b;
        hbw[c] = dt * rho * cc;
        if (fbx) fbx[c] += dt * a;
        if (fby) fby[c] += dt * b;
        if (fbz) fbz[c] += dt * cc;
    }
}

// u-bar += dt/Re L^T q + J_A(u^n)^T Hb (one component per call of the
// helpers below); p-bar -= dt G^T q.
// The window of one grid row (j, k) read by the two gather kernels: every
// value lies within one cell of (i, j, k) in each direction, so the row
// offsets of (j + dj, k + dk) (-1 beyond a wall) are formed once per block
// and the wrapped columns i - 1, i, i + 1 once per thread; the accessors take
// the offsets (di, dj, dk) in -1 .. 1.
struct Window {
    int nx, ny, nz, j, k;
    bool walls;
    int ro[3][3];   // [dj + 1][dk + 1]
    FSEI_D Window(const GridDev &g, int j_, int k_)
        : nx(g.nx), ny(g.ny), nz(g.nz), j(j_), k(k_), walls(g.walls != 0) {
        const Nb N{g.nx, g.ny, g.nz, g.walls};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const int kk = k + b - 1;
                ro[a][b] = N.zin(kk) ? (N.wzi(kk) * ny + N.wyi(j + a - 1)) * nx : -1;
            }
    }
    // the face k + dk is a wall face or lies beyond one
    FSEI_D bool wallface(int dk) const { return walls && (k + dk <= 0 || k + dk >= nz); }
    FSEI_D int zw(int kk) const { return kk < 0 ? kk + nz : (kk >= nz ? kk - nz : kk); }
};

// Pass 1 of the gather: the cotangents of the advection fluxes at the cell
// centres (Qb, Rb, Sb) and edges (Euv, Euw, Evw) from H-bar, each formed
// once per point (pass 2 reads each of them at up to eight points).
template <typename T>
__global__ void __launch_bounds__(256)
k_adj_flux(GridDev g, const T *__restrict__ H0, const T *__restrict__ H1,
           const T *__restrict__ H2, T *__restrict__ fl) {
    const Window Wn(g, blockIdx.x % g.ny, blockIdx.x / g.ny);
    const int nx = g.nx, k = Wn.k;
    const size_t ncell = (size_t)g.nx * g.ny * g.nz;
    const T idx = fpick<T>(g.idx, g.fidx), idy = fpick<T>(g.idy, g.fidy);
    const T *idz = Metric<T>::idz(g), *ihc = Metric<T>::ihc(g);
    auto IDZ = [&](int dk) { return idz[Wn.zw(k + dk)]; };
    auto IHC = [&](int dk) {
        const int kk = k + dk;
        return ihc[kk < 0 ? kk + Wn.nz : (kk > Wn.nz ? kk - Wn.nz : kk)];
    };
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int cm = i == 0 ? nx - 1 : i - 1, cp = i == nx - 1 ? 0 : i + 1;
        auto at = [&](const T *f, int di, int dj, int dk) {
            const int o = Wn.ro[dj + 1][dk + 1];
            return o < 0 ? T(0) : f[o + (di < 0 ? cm : (di > 0 ? cp : i))];
        };
        // cotangents of the advection term, with the sign of -div(uu) folded in
        auto A = [&](int di, int dj, int dk) { return -at(H0, di, dj, dk); };
        auto B = [&](int di, int dj, int dk) { return -at(H1, di, dj, dk); };
        auto C = [&](int di, int dj, int dk) {
            if (Wn.wallface(dk)) return T(0);
            return -at(H2, di, dj, dk);
        };
        const size_t c = fid(i, Wn.j, k, g.nx, g.ny);
        // Qb, Rb, Sb at the centre; Euv, Euw, Evw at the edges of (i, j, k)
        fl[c] = (A(0, 0, 0) - A(1, 0, 0)) * idx;
        fl[ncell + c] = (B(0, 0, 0) - B(0, 1, 0)) * idy;
        fl[2 * ncell + c] = C(0, 0, 0) * IHC(0) - C(0, 0, 1) * IHC(1);
        fl[3 * ncell + c] = (A(0, -1, 0) - A(0, 0, 0)) * idy + (B(-1, 0, 0) - B(0, 0, 0)) * idx;
        fl[4 * ncell + c] = Wn.wallface(0) ? T(0)
                                           : (A(0, 0, -1) * IDZ(-1) - A(0, 0, 0) * IDZ(0)) +
                                                 (C(-1, 0, 0) - C(0, 0, 0)) * idx;
        fl[5 * ncell + c] = Wn.wallface(0) ? T(0)
                                           : (B(0, 0, -1) * IDZ(-1) - B(0, 0, 0) * IDZ(0)) +
                                                 (C(0, -1, 0) - C(0, 0, 0)) * idy;
    }
}

// Pass 2: u-bar += dt/Re L^T q + J_A(u^n)^T Hb from the flux cotangents of
// pass 1 and the forward velocities; p-bar -= dt G^T q.
template <typename T>
__global__ void __launch_bounds__(256)
k_adj_gather(GridDev g, const T *__restrict__ u, const T *__restrict__ v,
             const T *__restrict__ w, const T *__restrict__ q0, const T *__restrict__ q1,
             const T *__restrict__ q2, const T *__restrict__ fl, T *__restrict__ ub,
             T *__restrict__ vb, T *__restrict__ wb, T *__restrict__ pb, const StepScalars *sc,
             T inv_re) {
    const Window Wn(g, blockIdx.x % g.ny, blockIdx.x / g.ny);
    const int nx = g.nx, nz = g.nz, j = Wn.j, k = Wn.k;
    const bool walls = Wn.walls;
    const size_t ncell = (size_t)g.nx * g.ny * g.nz;
    const T dt = fpick<T>(sc->dt, sc->fdt);
    const T idx = fpick<T>(g.idx, g.fidx), idy = fpick<T>(g.idy, g.fidy);
    const T idx2 = fpick<T>(g.idx2, g.fidx2), idy2 = fpick<T>(g.idy2, g.fidy2);
    const T *idz = Metric<T>::idz(g), *ihc = Metric<T>::ihc(g), *dz = Metric<T>::dz(g);
    const T h = T(0.5);
    auto IDZ = [&](int dk) { return idz[Wn.zw(k + dk)]; };
    auto wallface = [&](int dk) { return Wn.wallface(dk); };
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int cm = i == 0 ? nx - 1 : i - 1, cp = i == nx - 1 ? 0 : i + 1;
        auto at = [&](const T *f, int di, int dj, int dk) {
            const int o = Wn.ro[dj + 1][dk + 1];
            return o < 0 ? T(0) : f[o + (di < 0 ? cm : (di > 0 ? cp : i))];
        };
        // the flux cotangents of pass 1 (0 beyond a wall, as there)
        auto Qb = [&](int di, int dj, int dk) { return at(fl, di, dj, dk); };
        auto Rb = [&](int di, int dj, int dk) { return at(fl + ncell, di, dj, dk); };
        auto Sb = [&](int di, int dj, int dk) { return at(fl + 2 * ncell, di, dj, dk); };
        auto Euv = [&](int di, int dj, int dk) { return at(fl + 3 * ncell, di, dj, dk); };
        auto Euw = [&](int di, int dj, int dk) { return at(fl + 4 * ncell, di, dj, dk); };
        auto Evw = [&](int di, int dj, int dk) { return at(fl + 5 * ncell, di, dj, dk); };
        // forward averages
        auto U = [&](int di, int dj, int dk) { return at(u, di, dj, dk); };
        auto V = [&](int di, int dj, int dk) { return at(v, di, dj, dk); };
        auto Wf = [&](int di, int dj, int dk) {
            if (wallface(dk)) return T(0);
            return at(w, di, dj, dk);
        };
        const size_t c = fid(i, j, k, g.nx, g.ny);
        // ---- u
        {
            const T uc0 = h * (U(0, 0, 0) + U(1, 0, 0));
            const T ucm = h * (U(-1, 0, 0) + U(0, 0, 0));
            T a = h * (T(2) * uc0 * Qb(0, 0, 0) + T(2) * ucm * Qb(-1, 0, 0));
            a += h * (Euv(0, 0, 0) * h * (V(0, 0, 0) + V(-1, 0, 0)) +
                      Euv(0, 1, 0) * h * (V(0, 1, 0) + V(-1, 1, 0)));
            a += h * (Euw(0, 0, 0) * h * (Wf(0, 0, 0) + Wf(-1, 0, 0)) +
                      Euw(0, 0, 1) * h * (Wf(0, 0, 1) + Wf(-1, 0, 1)));
            // viscous: lap_xy(q) + dz_k lapz_centre(q / dz)
            const T qc = at(q0, 0, 0, 0);
            const T lxy = (at(q0, 1, 0, 0) - T(2) * qc + at(q0, -1, 0, 0)) * idx2 +
                          (at(q0, 0, 1, 0) - T(2) * qc + at(q0, 0, -1, 0)) * idy2;
            const T sq = qc * idz[k];
            const T sup = Wn.ro[1][2] >= 0 ? at(q0, 0, 0, 1) * IDZ(1) : T(0);
            const T sdn = Wn.ro[1][0] >= 0 ? at(q0, 0, 0, -1) * IDZ(-1) : T(0);
            const T lz = ((sup - sq) * ihc[k + 1] - (sq - sdn) * ihc[k]) * idz[k];
            ub[c] = ub[c] + dt * inv_re * (lxy + dz[k] * lz) + a;
        }
        // ---- v
        {
            const T vc0 = h * (V(0, 0, 0) + V(0, 1, 0));
            const T vcm = h * (V(0, -1, 0) + V(0, 0, 0));
            T a = h * (T(2) * vc0 * Rb(0, 0, 0) + T(2) * vcm * Rb(0, -1, 0));
            a += h * (Euv(0, 0, 0) * h * (U(0, 0, 0) + U(0, -1, 0)) +
                      Euv(1, 0, 0) * h * (U(1, 0, 0) + U(1, -1, 0)));
            a += h * (Evw(0, 0, 0) * h * (Wf(0, 0, 0) + Wf(0, -1, 0)) +
                      Evw(0, 0, 1) * h * (Wf(0, 0, 1) + Wf(0, -1, 1)));
            const T qc = at(q1, 0, 0, 0);
            const T lxy = (at(q1, 1, 0, 0) - T(2) * qc + at(q1, -1, 0, 0)) * idx2 +
                          (at(q1, 0, 1, 0) - T(2) * qc + at(q1, 0, -1, 0)) * idy2;
            const T sq = qc * idz[k];
            const T sup = Wn.ro[1][2] >= 0 ? at(q1, 0, 0, 1) * IDZ(1) : T(0);
            const T sdn = Wn.ro[1][0] >= 0 ? at(q1, 0, 0, -1) * IDZ(-1) : T(0);
            const T lz = ((sup - sq) * ihc[k + 1] - (sq - sdn) * ihc[k]) * idz[k];
            vb[c] = vb[c] + dt * inv_re * (lxy + dz[k] * lz) + a;
        }
        // ---- w
        if (walls && k == 0) {
            wb[c] = T(0);
        } else {
            const T wc0 = h * (Wf(0, 0, 0) + Wf(0, 0, 1));
            const T wcm = h * (Wf(0, 0, -1) + Wf(0, 0, 0));
            T a = h * (T(2) * wc0 * Sb(0, 0, 0) + T(2) * wcm * Sb(0, 0, -1));
            a += h * (Euw(0, 0, 0) * h * (U(0, 0, 0) + U(0, 0, -1)) +
                      Euw(1, 0, 0) * h * (U(1, 0, 0) + U(1, 0, -1)));
            a += h * (Evw(0, 0, 0) * h * (V(0, 0, 0) + V(0, 0, -1)) +
                      Evw(0, 1, 0) * h * (V(0, 1, 0) + V(0, 1, -1)));
            // viscous: lap_xy(q) + hc_k lapz_face(q / hc), q = 0 on the walls
            auto QW = [&](int di, int dj, int dk) {
                if (wallface(dk)) return T(0);
                return at(q2, di, dj, dk);
            };
            const T qc = QW(0, 0, 0);
            const T lxy = (QW(1, 0, 0) - T(2) * qc + QW(-1, 0, 0)) * idx2 +
                          (QW(0, 1, 0) - T(2) * qc + QW(0, -1, 0)) * idy2;
            const T sq = qc * ihc[k];
            const T sup = QW(0, 0, 1) * ihc[k + 1 == nz ? (walls ? nz : 0) : k + 1];
            const T sdn = QW(0, 0, -1) * ihc[k - 1 < 0 ? nz - 1 : k - 1];
            const T lz = ((sup - sq) * idz[k] - (sq - sdn) * IDZ(-1)) * ihc[k];
            wb[c] = wb[c] + dt * inv_re * (lxy + lz / ihc[k]) + a;
        }
        // ---- p: p-bar -= dt G^T q
        {
            const T cz0 = (walls && k == 0) ? T(0) : at(q2, 0, 0, 0) * ihc[k];
            const T cz1 = (walls && k == nz - 1) ? T(0) : at(q2, 0, 0, 1) * ihc[k + 1];
            const T gtq = (at(q0, 0, 0, 0) - at(q0, 1, 0, 0)) * idx +
                          (at(q1, 0, 0, 0) - at(q1, 0, 1, 0)) * idy + (cz0 - cz1);
            pb[c] = pb[c] - dt * gtq;
        }
    }
}

// (I - beta L_x)^-1 of q0, q1, q2 row by row, the row-resident layout of the
// forward RHS (LPR lanes per row, 4 cells per lane in registers, rpb rows
// per block) and its register line solve: the x operator is symmetric, so
// the adjoint x sweep is the forward one without the right-hand side.
template <typename T, int LPR>
__global__ void __launch_bounds__(LPR > 128 ? LPR : 128)
k_sweep_x_row(GridDev g, T *__restrict__ q0, T *__restrict__ q1, T *__restrict__ q2,
              const StepScalars *sc, int rpb) {
    constexpr int CPL = 4;
    __shared__ T xs[LPR > 32 ? 2 * 3 * (LPR > 128 ? LPR : 128) : 1];
    const int nx = g.nx, ny = g.ny;
    const int nby = ny / rpb;
    const int k = blockIdx.x / nby;
    const int j = (blockIdx.x % nby) * rpb + (int)threadIdx.x / LPR;
    const size_t o = ((size_t)k * ny + j) * nx + ((int)threadIdx.x & (LPR - 1)) * CPL;
    T R[3][CPL];
    ldrow(R[0], q0 + o);
    ldrow(R[1], q1 + o);
    ldrow(R[2], q2 + o);
    line_solve_uni<T, CPL, LPR, 3>(R, fpick<T>(sc->ax, sc->fax), fpick<T>(sc->cix, sc->fcix),
                                   sizeof(T) == 4 ? sc->ndecx_f : sc->ndecx_d, xs);
    strow(q0 + o, R[0]);
    strow(q1 + o, R[1]);
    strow(q2 + o, R[2]);
}

template <typename T, int LPR>
void sweep_x_row_launch(const GridDev &g, Work<T> &W, const StepScalars *sc, int rpb,
                        cudaStream_t st) {
    k_sweep_x_row<T, LPR><<<g.nz * (g.ny / rpb), rpb * LPR, 0, st>>>(g, W.q0, W.q1, W.q2, sc, rpb);
}

// the row-resident adjoint x sweep where rows split into lanes of 4 cells
template <typename T>
bool sweep_x_row_any(const GridDev &g, Work<T> &W, const StepScalars *sc, cudaStream_t st) {
    int cpl = 0, lpr = 0, rpb = 0;
    if (!rhs_row_geometry<T>(g, cpl, lpr, rpb, 4) || cpl != 4) return false;
    switch (lpr) {
    case 4: sweep_x_row_launch<T, 4>(g, W, sc, rpb, st); return true;
    case 8: sweep_x_row_launch<T, 8>(g, W, sc, rpb, st); return true;
    case 16: sweep_x_row_launch<T, 16>(g, W, sc, rpb, st); return true;
    case 32: sweep_x_row_launch<T, 32>(g, W, sc, rpb, st); return true;
    case 64: sweep_x_row_launch<T, 64>(g, W, sc, rpb, st); return true;
    case 128: sweep_x_row_launch<T, 128>(g, W, sc, rpb, st); return true;
    case 256: sweep_x_row_launch<T, 256>(g, W, sc, rpb, st); return true;
    default: return false;
    }
}

}  // namespace

// chunks per line of the adjoint x sweep (ry lines per block, 256 threads)
template <typename T> void sweep_x_geometry(const GridDev &g, const Work<T> &W, int &P, int &chunk) {
    uni_geometry(g.nx, W.ry, 256, P, chunk);
}

template <typename T, int L>
void sweep_x_L(const GridDev &g, Work<T> &W, const StepScalars *sc, int P, cudaStream_t st) {
    const int ry = W.ry;
    const int threads = ((ry * P + 31) / 32) * 32;
    const size_t smem = sizeof(T) * ((size_t)g.nx * (ry | 1) + 2 * (size_t)ry * P);
    k_sweep_x<T, L><<<3 * g.nz * (g.ny / ry), threads < 64 ? 64 : threads, smem, st>>>(
        g, W.q0, W.q1, W.q2, sc, ry, P);
}

template <typename T>
void launch_sweep_x_adjoint(const GridDev &g, Work<T> &W, const StepScalars *sc, cudaStream_t st) {
    if (sweep_x_row_any<T>(g, W, sc, st)) return;
    int P, chunk;
    sweep_x_geometry(g, W, P, chunk);
    if (chunk <= 8) sweep_x_L<T, 8>(g, W, sc, P, st);
    else if (chunk <= 16) sweep_x_L<T, 16>(g, W, sc, P, st);
    else if (chunk <= 32) sweep_x_L<T, 32>(g, W, sc, P, st);
    else sweep_x_L<T, 64>(g, W, sc, P, st);
}

template <typename T>
void launch_adjoint_step(const GridDev &g, Work<T> &W, StepScalars *sc, const T *u, const T *v,
                         const T *w, T *ub, T *vb, T *wb, T *pb, T *hbu, T *hbv, T *hbw, T *fbx,
                         T *fby, T *fbz, double re, cudaStream_t st, const LaunchHook *hook) {
    const int rows = g.ny * g.nz;
    const int thr = g.nx >= 256 ? 256 : ((g.nx + 31) / 32) * 32;
    auto group = [&](int kind, auto &&launch) {
        if (hook) hook->before(hook->ctx, kind, st);
        launch();
        if (hook) hook->after(hook->ctx, kind, st);
    };
    group(AK_PHIBAR, [&] { k_adj_phibar<T><<<rows, thr, 0, st>>>(g, ub, vb, wb, pb, W.phi, sc); });
    group(AK_POISSON, [&] {
        launch_rfft_x<T>(g, W, sc, W.phi, 1, st);
        launch_fft_y<T>(g, W, 0, st);
        launch_poisson_z<T>(g, W, st, 1);
        launch_fft_y<T>(g, W, 1, st);
        launch_irfft_x<T>(g, W, W.phi, st);
    });
    group(AK_USTAR, [&] {
        k_adj_ustar<T><<<rows, thr, 0, st>>>(g, ub, vb, wb, W.phi, W.q0, W.q1, W.q2, sc);
    });
    group(AK_SWEEP_Z, [&] { launch_sweep_z_adjoint<T>(g, W, st); });
    group(AK_SWEEP_Y, [&] { launch_sweep_y<T>(g, W, sc, st); });
    group(AK_SWEEP_X, [&] { launch_sweep_x_adjoint<T>(g, W, sc, st); });
    group(AK_HIST, [&] {
        k_adj_hist<T><<<rows, thr, 0, st>>>(g, W.q0, W.q1, W.q2, hbu, hbv, hbw, W.adj0, W.adj1,
                                            W.adj2, fbx, fby, fbz, sc);
    });
    group(AK_GATHER, [&] {
        k_adj_flux<T><<<rows, thr, 0, st>>>(g, W.adj0, W.adj1, W.adj2, W.adjf);
        k_adj_gather<T><<<rows, thr, 0, st>>>(g, u, v, w, W.q0, W.q1, W.q2, W.adjf, ub, vb, wb,
                                              pb, sc, T(1.0 / re));
    });
}

template <typename T> void set_smem_limits_adjoint(const GridDev &g, const Work<T> &W) {
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_adj_phibar<T>);
    cudaFuncGetAttributes(&fa, k_adj_ustar<T>);
    cudaFuncGetAttributes(&fa, k_adj_hist<T>);
    cudaFuncGetAttributes(&fa, k_adj_flux<T>);
    cudaFuncGetAttributes(&fa, k_adj_gather<T>);
    raise_smem_limit(k_sweep_x<T, 8>);
    raise_smem_limit(k_sweep_x<T, 16>);
    raise_smem_limit(k_sweep_x<T, 32>);
    raise_smem_limit(k_sweep_x<T, 64>);
}

#define FSEI_INST(T)                                                                           \
    template void launch_adjoint_step<T>(const GridDev &, Work<T> &, StepScalars *, const T *,  \
                                         const T *, const T *, T *, T *, T *, T *, T *, T *,    \
                                         T *, T *, T *, T *, double, cudaStream_t,              \
                                         const LaunchHook *);                                   \
    template void set_smem_limits_adjoint<T>(const GridDev &, const Work<T> &);
FSEI_INST(float)
FSEI_INST(double)
#undef FSEI_INST

}  // namespace fsei
