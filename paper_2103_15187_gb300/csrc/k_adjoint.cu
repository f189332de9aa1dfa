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
//   k_adj_gather_tile
//                  u-bar = u*-bar + dt/Re L^T q + J_A(u^n)^T Hb;
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
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int j = blockIdx.x % ny, k = blockIdx.x / ny;
    const bool walls = g.walls != 0;
    const T dt = fpick<T>(sc->dt, sc->fdt), beta = fpick<T>(sc->beta, sc->fbeta);
    const T idx = fpick<T>(g.idx, g.fidx), idy = fpick<T>(g.idy, g.fidy);
    const T idx2 = fpick<T>(g.idx2, g.fidx2), idy2 = fpick<T>(g.idy2, g.fidy2);
    const T *idz = Metric<T>::idz(g), *ihc = Metric<T>::ihc(g), *dz = Metric<T>::dz(g);
    const int kd = k == 0 ? nz - 1 : k - 1, ku = k == nz - 1 ? 0 : k + 1;
    const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
    // 32-bit offsets of the rows (j, k), (j -/+ 1, k), (j, k -/+ 1) and the
    // metric values of plane k, once per block (the planes beyond a wall
    // are never read)
    const int oc = (k * ny + j) * nx, ojm = (k * ny + jm) * nx, ojp = (k * ny + jp) * nx;
    const int okd = (kd * ny + j) * nx, oku = (ku * ny + j) * nx;
    const bool bot = walls && k == 0, top = walls && k == nz - 1;
    const T ihck = ihc[k], ihcu = ihc[k + 1], idzk = idz[k], idzd = idz[kd], idzu = idz[ku];
    const T dzk = dz[k];
    const T inv_vol = T(g.idx * g.idy) * idzk;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int im = i == 0 ? nx - 1 : i - 1, ip = i == nx - 1 ? 0 : i + 1;
        // G^T u-bar
        const T cz0 = bot ? T(0) : wb[oc + i] * ihck;
        const T cz1 = top ? T(0) : wb[oku + i] * ihcu;
        const T gtu = (ub[oc + i] - ub[oc + ip]) * idx + (vb[oc + i] - vb[ojp + i]) * idy +
                      (cz0 - cz1);
        // (DG)^T p-bar = lap_xy(p-bar) + dz_k lapz((p-bar) / dz)
        const T p0 = pb[oc + i];
        const T lxy = (pb[oc + ip] - T(2) * p0 + pb[oc + im]) * idx2 +
                      (pb[ojp + i] - T(2) * p0 + pb[ojm + i]) * idy2;
        const T q0 = p0 * idzk;
        const T fup = top ? T(0) : (pb[oku + i] * idzu - q0) * ihcu;
        const T fdn = bot ? T(0) : (q0 - pb[okd + i] * idzd) * ihck;
        const T lp = lxy + dzk * (fup - fdn) * idzk;
        const T phib = -dt * gtu + p0 - beta * lp;
        x[oc + i] = phib * inv_vol;
    }
}

// The same with 16-byte vectors: a thread owns W = 16 / sizeof(T)
// consecutive cells of a row (x neighbours beyond its vector as scalars), a
// block of 256 threads covers 256 W / nx rows of plane k.  The arithmetic of
// each cell is that of k_adj_phibar, in the same order.  Needs nx % W == 0.
template <typename T>
__global__ void __launch_bounds__(256)
k_adj_phibar_vec(GridDev g, const T *__restrict__ ub, const T *__restrict__ vb,
                 const T *__restrict__ wb, const T *__restrict__ pb, T *__restrict__ x,
                 const StepScalars *sc) {
    using V = Vec16<T>;
    constexpr int W = V::W;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int tpr = nx / W, rpb = (int)blockDim.x / tpr;
    const int nbj = (ny + rpb - 1) / rpb;
    const int k = blockIdx.x / nbj;
    const int j = (blockIdx.x % nbj) * rpb + (int)threadIdx.x / tpr;
    const int i0 = ((int)threadIdx.x % tpr) * W;
    if (j >= ny || (int)threadIdx.x >= tpr * rpb) return;
    const bool walls = g.walls != 0;
    const T dt = fpick<T>(sc->dt, sc->fdt), beta = fpick<T>(sc->beta, sc->fbeta);
    const T idx = fpick<T>(g.idx, g.fidx), idy = fpick<T>(g.idy, g.fidy);
    const T idx2 = fpick<T>(g.idx2, g.fidx2), idy2 = fpick<T>(g.idy2, g.fidy2);
    const T *idz = Metric<T>::idz(g), *ihc = Metric<T>::ihc(g), *dz = Metric<T>::dz(g);
    const int kd = k == 0 ? nz - 1 : k - 1, ku = k == nz - 1 ? 0 : k + 1;
    const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
    const int oc = (k * ny + j) * nx, ojm = (k * ny + jm) * nx, ojp = (k * ny + jp) * nx;
    const int okd = (kd * ny + j) * nx, oku = (ku * ny + j) * nx;
    const bool bot = walls && k == 0, top = walls && k == nz - 1;
    const T ihck = ihc[k], ihcu = ihc[k + 1], idzk = idz[k], idzd = idz[kd], idzu = idz[ku];
    const T dzk = dz[k];
    const T inv_vol = T(g.idx * g.idy) * idzk;
    auto ld = [](const T *p) { return *reinterpret_cast<const V *>(p); };
    const int iw = i0 + W == nx ? 0 : i0 + W, im0 = i0 == 0 ? nx - 1 : i0 - 1;
    const V u0 = ld(ub + oc + i0), v0 = ld(vb + oc + i0), v1 = ld(vb + ojp + i0);
    const V p0 = ld(pb + oc + i0), pjp = ld(pb + ojp + i0), pjm = ld(pb + ojm + i0);
    V w0, w1, pku, pkd;
    if (!bot) { w0 = ld(wb + oc + i0); pkd = ld(pb + okd + i0); }
    if (!top) { w1 = ld(wb + oku + i0); pku = ld(pb + oku + i0); }
    const T uW = ub[oc + iw], pW = pb[oc + iw], pM = pb[oc + im0];
    V out;
#pragma unroll
    for (int e = 0; e < W; ++e) {
        const T up = e == W - 1 ? uW : u0.v[e + 1];
        const T pp = e == W - 1 ? pW : p0.v[e + 1];
        const T pm = e == 0 ? pM : p0.v[e - 1];
        // G^T u-bar
        const T cz0 = bot ? T(0) : w0.v[e] * ihck;
        const T cz1 = top ? T(0) : w1.v[e] * ihcu;
        const T gtu = (u0.v[e] - up) * idx + (v0.v[e] - v1.v[e]) * idy + (cz0 - cz1);
        // (DG)^T p-bar = lap_xy(p-bar) + dz_k lapz((p-bar) / dz)
        const T pc = p0.v[e];
        const T lxy = (pp - T(2) * pc + pm) * idx2 + (pjp.v[e] - T(2) * pc + pjm.v[e]) * idy2;
        const T q0 = pc * idzk;
        const T fup = top ? T(0) : (pku.v[e] * idzu - q0) * ihcu;
        const T fdn = bot ? T(0) : (q0 - pkd.v[e] * idzd) * ihck;
        const T lp = lxy + dzk * (fup - fdn) * idzk;
        const T phib = -dt * gtu + pc - beta * lp;
        out.v[e] = phib * inv_vol;
    }
    *reinterpret_cast<V *>(x + oc + i0) = out;
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

// The gather in one pass, tiled and marched along z: a block owns a tile of
// TX x TY columns (i, j) and walks a chunk of consecutive planes k.  The nine
// fields the gather reads around a cell -- H-bar (H0, H1, H2), u^n, v^n, w^n
// and q0, q1, q2 -- are staged plane by plane in shared memory on the tile
// extended by one column and one row on every side (x, y periodic, wrapped
// by global index), in a ring of NS planes: the planes k - 1, k, k + 1 the
// cell needs and the NS - 3 planes after them, copied with cp.async while
// plane k is computed.  Planes beyond a wall are staged as zeros, and the
// wall faces too for the face fields (H2, w, q2), which is what the
// two-pass formulation reads there.  Each cell evaluates the flux
// cotangents it needs (at most nine points of the 3 x 3 x 3 window) from the
// staged H-bar directly -- the cotangents of the advection fluxes at the
// cell centres (Qb, Rb, Sb) and edges (Euv, Euw, Evw) -- then
//   u-bar += dt/Re L^T q + J_A(u^n)^T Hb,   p-bar -= dt G^T q,
// so no flux field goes through global memory.  The cotangents it updates
// and the plane's metric values are read before the wait for the staged
// planes, so their latency overlaps it.
enum GatherField { GF_H0, GF_H1, GF_H2, GF_U, GF_V, GF_W, GF_Q0, GF_Q1, GF_Q2, GF_COUNT };

template <int TX, int TY> constexpr int gather_plane() { return (TX + 2) * (TY + 2); }

// Single precision: 4 blocks of 256 per SM with four planes in the ring (63
// registers, no spills; at 128 x 128 x 192 92 us against 96 us for five
// planes at 3 blocks); double precision: 2 (the ring takes 98 KB).
template <typename T, int NS> constexpr int gather_min_blocks() {
    return sizeof(T) == 4 ? (NS == 4 ? 4 : 3) : 2;
}

template <typename T, int TX, int TY, int NS>
__global__ void __launch_bounds__(TX * TY, (gather_min_blocks<T, NS>()))
k_adj_gather_tile(GridDev g, const T *__restrict__ u, const T *__restrict__ v,
                  const T *__restrict__ w, const T *__restrict__ q0, const T *__restrict__ q1,
                  const T *__restrict__ q2, const T *__restrict__ H0, const T *__restrict__ H1,
                  const T *__restrict__ H2, T *__restrict__ ub, T *__restrict__ vb,
                  T *__restrict__ wb, T *__restrict__ pb, const StepScalars *sc, T inv_re,
                  int kc) {
    static_assert(NS == 4 || NS == 5, "ring of 4 or 5 planes");
    constexpr int LEAD = NS - 3;
    extern __shared__ __align__(16) unsigned char gather_smem[];
    T *const sm = reinterpret_cast<T *>(gather_smem);
    constexpr int PW = TX + 2, PL = gather_plane<TX, TY>(), SLOT = GF_COUNT * PL;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const bool walls = g.walls != 0;
    const int tx = (int)threadIdx.x % TX, ty = (int)threadIdx.x / TX;
    const int i0 = (int)blockIdx.x * TX, j0 = (int)blockIdx.y * TY;
    const int k0 = (int)blockIdx.z * kc, k1 = min(k0 + kc, nz);
    const int i = i0 + tx, j = j0 + ty;
    const bool mine = i < nx && j < ny;
    const T *const src[GF_COUNT] = {H0, H1, H2, u, v, w, q0, q1, q2};
    // ring slot of plane kk (kk >= -1)
    auto slot = [](int kk) { return NS == 4 ? (kk & 3) : (kk + NS) % NS; };
    // copies of plane kk (wrapped, or zeros beyond a wall) into its slot
    auto stage = [&](int kk) {
        T *d = sm + slot(kk) * SLOT;
        const bool out = walls && (kk < 0 || kk >= nz);
        const bool face0 = walls && (kk <= 0 || kk >= nz);
        const int kw = kk < 0 ? kk + nz : (kk >= nz ? kk - nz : kk);
        for (int e = threadIdx.x; e < PL; e += TX * TY) {
            const int r = e / PW, c = e - r * PW;
            int gj = j0 + r - 1, gi = i0 + c - 1;
            gj = gj < 0 ? gj + ny : (gj >= ny ? gj % ny : gj);
            gi = gi < 0 ? gi + nx : (gi >= nx ? gi % nx : gi);
            const size_t o = ((size_t)kw * ny + gj) * nx + gi;
#pragma unroll
            for (int f = 0; f < GF_COUNT; ++f) {
                const bool face = f == GF_H2 || f == GF_W || f == GF_Q2;
                T *dst = d + f * PL + e;
                if (face ? face0 : out) {
                    *dst = T(0);
                } else if constexpr (sizeof(T) == 8) {
                    cp_async8(dst, src[f] + o);
                } else {
                    cp_async4(dst, src[f] + o);
                }
            }
        }
    };
    const T dt = fpick<T>(sc->dt, sc->fdt);
    const T idx = fpick<T>(g.idx, g.fidx), idy = fpick<T>(g.idy, g.fidy);
    const T idx2 = fpick<T>(g.idx2, g.fidx2), idy2 = fpick<T>(g.idy2, g.fidy2);
    const T *idz = Metric<T>::idz(g), *ihc = Metric<T>::ihc(g), *dz = Metric<T>::dz(g);
    const T h = T(0.5);
    const int me = (ty + 1) * PW + tx + 1;
    stage(k0 - 1);
    stage(k0);
    stage(k0 + 1);
    cp_async_commit();
#pragma unroll
    for (int l = 1; l < LEAD; ++l) {
        if (k0 + 1 + l <= k1) stage(k0 + 1 + l);
        cp_async_commit();
    }
    for (int k = k0; k < k1; ++k) {
        const size_t c = ((size_t)k * ny + j) * nx + i;
        // the cotangents this cell updates and the metric values of plane k
        T ub0 = T(0), vb0 = T(0), wb0 = T(0), pb0 = T(0);
        if (mine) {
            ub0 = ub[c];
            vb0 = vb[c];
            wb0 = wb[c];
            pb0 = pb[c];
        }
        const int kmw = k == 0 ? nz - 1 : k - 1, kpw = k == nz - 1 ? 0 : k + 1;
        const T idzk = idz[k], idzm = idz[kmw], idzp = idz[kpw], dzk = dz[k];
        const T ihck = ihc[k], ihcp = ihc[k + 1], ihcm = ihc[kmw];
        const T ihcw = ihc[k + 1 == nz ? (walls ? nz : 0) : k + 1];
        if (LEAD == 1) cp_async_wait_all();
        else cp_async_wait_prior();
        __syncthreads();           // plane k + 1 landed; the slot of k - 2 is free
        if (k + 1 + LEAD <= k1) stage(k + 1 + LEAD);
        cp_async_commit();
        const T *const P[3] = {sm + slot(k - 1) * SLOT + me, sm + slot(k) * SLOT + me,
                               sm + slot(k + 1) * SLOT + me};
        // the staged value of field f at (i + di, j + dj, k + dk)
        auto S = [&](int f, int di, int dj, int dk) { return P[dk + 1][f * PL + dj * PW + di]; };
        // idz of the plane k + dk (dk in -2 .. 1), wrapped
        auto IDZ = [&](int dk) {
            return dk == 0 ? idzk : (dk == 1 ? idzp : (dk == -1 ? idzm : idz[(k - 2 + 2 * nz) % nz]));
        };
        auto wallface = [&](int dk) { return walls && (k + dk <= 0 || k + dk >= nz); };
        // advection cotangents with the sign of -div(uu) folded in (wall
        // faces of H2 are staged as 0)
        auto A = [&](int di, int dj, int dk) { return -S(GF_H0, di, dj, dk); };
        auto B = [&](int di, int dj, int dk) { return -S(GF_H1, di, dj, dk); };
        auto C = [&](int di, int dj, int dk) { return -S(GF_H2, di, dj, dk); };
        // flux cotangents at the point (i + di, j + dj, k + dk)
        auto Qb = [&](int di, int dj, int dk) {
            return (A(di, dj, dk) - A(di + 1, dj, dk)) * idx;
        };
        auto Rb = [&](int di, int dj, int dk) {
            return (B(di, dj, dk) - B(di, dj + 1, dk)) * idy;
        };
        // Sb at the point k (dk = 0) or k - 1 (dk = -1; 0 below a wall)
        auto Sb = [&](int dk) {
            if (dk == 0) return C(0, 0, 0) * ihck - C(0, 0, 1) * ihcp;
            if (walls && k == 0) return T(0);
            return C(0, 0, -1) * ihc[k == 0 ? nz - 1 : k - 1] - C(0, 0, 0) * ihc[k == 0 ? nz : k];
        };
        auto Euv = [&](int di, int dj, int dk) {
            return (A(di, dj - 1, dk) - A(di, dj, dk)) * idy +
                   (B(di - 1, dj, dk) - B(di, dj, dk)) * idx;
        };
        auto Euw = [&](int di, int dj, int dk) {
            if (wallface(dk)) return T(0);
            return (A(di, dj, dk - 1) * IDZ(dk - 1) - A(di, dj, dk) * IDZ(dk)) +
                   (C(di - 1, dj, dk) - C(di, dj, dk)) * idx;
        };
        auto Evw = [&](int di, int dj, int dk) {
            if (wallface(dk)) return T(0);
            return (B(di, dj, dk - 1) * IDZ(dk - 1) - B(di, dj, dk) * IDZ(dk)) +
                   (C(di, dj - 1, dk) - C(di, dj, dk)) * idy;
        };
        auto U = [&](int di, int dj, int dk) { return S(GF_U, di, dj, dk); };
        auto V = [&](int di, int dj, int dk) { return S(GF_V, di, dj, dk); };
        auto Wf = [&](int di, int dj, int dk) { return S(GF_W, di, dj, dk); };
        if (mine) {
            // ---- u
            {
                const T uc0 = h * (U(0, 0, 0) + U(1, 0, 0));
                const T ucm = h * (U(-1, 0, 0) + U(0, 0, 0));
                T a = h * (T(2) * uc0 * Qb(0, 0, 0) + T(2) * ucm * Qb(-1, 0, 0));
                a += h * (Euv(0, 0, 0) * h * (V(0, 0, 0) + V(-1, 0, 0)) +
                          Euv(0, 1, 0) * h * (V(0, 1, 0) + V(-1, 1, 0)));
                a += h * (Euw(0, 0, 0) * h * (Wf(0, 0, 0) + Wf(-1, 0, 0)) +
                          Euw(0, 0, 1) * h * (Wf(0, 0, 1) + Wf(-1, 0, 1)));
                const T qc = S(GF_Q0, 0, 0, 0);
                const T lxy = (S(GF_Q0, 1, 0, 0) - T(2) * qc + S(GF_Q0, -1, 0, 0)) * idx2 +
                              (S(GF_Q0, 0, 1, 0) - T(2) * qc + S(GF_Q0, 0, -1, 0)) * idy2;
                const T sq = qc * idzk;
                const T sup = S(GF_Q0, 0, 0, 1) * idzp;
                const T sdn = S(GF_Q0, 0, 0, -1) * idzm;
                const T lz = ((sup - sq) * ihcp - (sq - sdn) * ihck) * idzk;
                ub[c] = ub0 + dt * inv_re * (lxy + dzk * lz) + a;
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
                const T qc = S(GF_Q1, 0, 0, 0);
                const T lxy = (S(GF_Q1, 1, 0, 0) - T(2) * qc + S(GF_Q1, -1, 0, 0)) * idx2 +
                              (S(GF_Q1, 0, 1, 0) - T(2) * qc + S(GF_Q1, 0, -1, 0)) * idy2;
                const T sq = qc * idzk;
                const T sup = S(GF_Q1, 0, 0, 1) * idzp;
                const T sdn = S(GF_Q1, 0, 0, -1) * idzm;
                const T lz = ((sup - sq) * ihcp - (sq - sdn) * ihck) * idzk;
                vb[c] = vb0 + dt * inv_re * (lxy + dzk * lz) + a;
            }
            // ---- w
            if (walls && k == 0) {
                wb[c] = T(0);
            } else {
                const T wc0 = h * (Wf(0, 0, 0) + Wf(0, 0, 1));
                const T wcm = h * (Wf(0, 0, -1) + Wf(0, 0, 0));
                T a = h * (T(2) * wc0 * Sb(0) + T(2) * wcm * Sb(-1));
                a += h * (Euw(0, 0, 0) * h * (U(0, 0, 0) + U(0, 0, -1)) +
                          Euw(1, 0, 0) * h * (U(1, 0, 0) + U(1, 0, -1)));
                a += h * (Evw(0, 0, 0) * h * (V(0, 0, 0) + V(0, 0, -1)) +
                          Evw(0, 1, 0) * h * (V(0, 1, 0) + V(0, 1, -1)));
                // viscous: lap_xy(q) + hc_k lapz_face(q / hc), q = 0 on the walls
                const T qc = S(GF_Q2, 0, 0, 0);
                const T lxy = (S(GF_Q2, 1, 0, 0) - T(2) * qc + S(GF_Q2, -1, 0, 0)) * idx2 +
                              (S(GF_Q2, 0, 1, 0) - T(2) * qc + S(GF_Q2, 0, -1, 0)) * idy2;
                const T sq = qc * ihck;
                const T sup = S(GF_Q2, 0, 0, 1) * ihcw;
                const T sdn = S(GF_Q2, 0, 0, -1) * ihcm;
                const T lz = ((sup - sq) * idzk - (sq - sdn) * idzm) * ihck;
                wb[c] = wb0 + dt * inv_re * (lxy + lz / ihck) + a;
            }
            // ---- p: p-bar -= dt G^T q
            {
                const T cz0 = (walls && k == 0) ? T(0) : S(GF_Q2, 0, 0, 0) * ihck;
                const T cz1 = (walls && k == nz - 1) ? T(0) : S(GF_Q2, 0, 0, 1) * ihcp;
                const T gtq = (S(GF_Q0, 0, 0, 0) - S(GF_Q0, 1, 0, 0)) * idx +
                              (S(GF_Q1, 0, 0, 0) - S(GF_Q1, 0, 1, 0)) * idy + (cz0 - cz1);
                pb[c] = pb0 - dt * gtq;
            }
        }
    }
    cp_async_wait_all();
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

// shared memory of k_adj_gather_tile: a ring of NS staged planes
template <typename T, int TX, int TY, int NS> constexpr size_t gather_smem_bytes() {
    return NS * (size_t)GF_COUNT * gather_plane<TX, TY>() * sizeof(T);
}

// planes per block of k_adj_gather_tile: chunks of at least 8 planes (the
// two extra planes each block stages cost at most a quarter more reads),
// as few as leave about four blocks per SM of work
inline int gather_chunk(const GridDev &g, int tx, int ty) {
    const long tiles = (long)((g.nx + tx - 1) / tx) * ((g.ny + ty - 1) / ty);
    const long want = 4L * 152;
    int kc = g.nz;
    while (kc > 8 && tiles * ((g.nz + kc - 1) / kc) < want) kc = (kc + 1) / 2;
    return kc < 8 ? (g.nz < 8 ? g.nz : 8) : kc;
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
    group(AK_PHIBAR, [&] {
        constexpr int VW = 16 / (int)sizeof(T);
        const int tpr = g.nx / VW;
        if (g.nx % VW == 0 && tpr <= 256) {
            const int rpb = 256 / tpr;
            const int blocks = g.nz * ((g.ny + rpb - 1) / rpb);
            k_adj_phibar_vec<T><<<blocks, 256, 0, st>>>(g, ub, vb, wb, pb, W.phi, sc);
        } else {
            k_adj_phibar<T><<<rows, thr, 0, st>>>(g, ub, vb, wb, pb, W.phi, sc);
        }
    });
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
        constexpr int TX = 32, TY = 8;
        const int kc = gather_chunk(g, TX, TY);
        const dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + kc - 1) / kc);
        k_adj_gather_tile<T, TX, TY, 4><<<grid, TX * TY, gather_smem_bytes<T, TX, TY, 4>(), st>>>(
            g, u, v, w, W.q0, W.q1, W.q2, W.adj0, W.adj1, W.adj2, ub, vb, wb, pb, sc, T(1.0 / re),
            kc);
    });
}

template <typename T> void set_smem_limits_adjoint(const GridDev &g, const Work<T> &W) {
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_adj_phibar<T>);
    cudaFuncGetAttributes(&fa, k_adj_ustar<T>);
    cudaFuncGetAttributes(&fa, k_adj_hist<T>);
    raise_smem_limit(k_adj_gather_tile<T, 32, 8, 4>);
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
