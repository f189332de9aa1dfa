// Explicit right-hand side and implicit viscous sweeps of one fractional
// step (Sec. 2.1, Eq. 3; Sec. 3.1 approximate factorisation with one
// tridiagonal system per direction, cyclic in x and y).
//
//   k_speed       max over cells of |u_c|/dx + |v_c|/dy + |w_c|/dz_k (for the
//                 CFL time step), double reduction
//   k_scalars     dt, beta = dt/(2 Re), gamma, rho of the step; resets the
//                 step's reductions
//   k_plans       matrix-only factors of the two z sweep matrices (centres,
//                 faces) for this step's beta; the uniform x and y lines need
//                 only alpha and 1/c of their cyclic Toeplitz factorisation,
//                 set by k_scalars
//   k_rhs_x       H^n = -div(uu)^n, RHS = dt[gamma H^n + rho H^{n-1}
//                 + Re^-1 L u^n - G p^n + f], stores H^n, solves
//                 (I - beta L_x) q = RHS along x (uni_solve)
// (the y and z sweeps are in k_lines.cu)
#include <string.h>

#include "kernels.cuh"
#include "rhs_row.cuh"
#include "tri.cuh"

namespace fsei {

namespace {

// one block per group of rows (no integer division per element); per-cell
// speed in the field precision, the grid-wide maximum in double
template <typename T>
FSEI_D void
k_speed(GridDev g, const T *__restrict__ u, const T *__restrict__ v, const T *__restrict__ w,
        StepScalars *sc, int rows) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int nbj = ny / rows;
    const int k = blockIdx.x / nbj, j0 = (blockIdx.x % nbj) * rows;
    const bool hasup = !g.walls || k < nz - 1;
    const int ku = k == nz - 1 ? 0 : k + 1;
    const T idx = fpick<T>(g.idx, g.fidx), idy = fpick<T>(g.idy, g.fidy);
    const T idzk = Metric<T>::idz(g)[k];
    T m = T(0);
    for (int r = 0; r < rows; ++r) {
        const int j = j0 + r, jp = j == ny - 1 ? 0 : j + 1;
        const size_t oc = ((size_t)k * ny + j) * nx;
        const T *ur = u + oc, *vr = v + oc, *vjp = v + ((size_t)k * ny + jp) * nx, *wr = w + oc,
                *wkur = w + ((size_t)ku * ny + j) * nx;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const int ip = i == nx - 1 ? 0 : i + 1;
            const T uc = T(0.5) * (ur[i] + ur[ip]);
            const T vc = T(0.5) * (vr[i] + vjp[i]);
            const T wku = hasup ? wkur[i] : T(0);
            const T wc = T(0.5) * (wr[i] + wku);
            m = fmax(m, fabs(uc) * idx + fabs(vc) * idy + fabs(wc) * idzk);
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    __shared__ double wmax[32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = (double)m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = 0.0;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) mm = fmax(mm, wmax[w]);
        atomicMax(&sc->speed_next, dbits(mm));
    }
}

// k_speed with 16-byte vectors: a thread owns VW = 16 / sizeof(T)
// consecutive cells of a row (the u neighbour beyond them as a scalar),
// tpr = nx / VW threads span a row, rpp = blockDim / tpr rows side by side;
// needs nx % VW == 0.  Same per-cell arithmetic as k_speed.
template <typename T>
FSEI_D void
k_speed_vec(GridDev g, const T *__restrict__ u, const T *__restrict__ v,
            const T *__restrict__ w, StepScalars *sc, int rows) {
    constexpr int VW = 16 / (int)sizeof(T);
    struct alignas(16) V { T x[VW]; };
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int tpr = nx / VW, nthr = (int)blockDim.x;
    const int rpp = tpr >= nthr ? 1 : nthr / tpr;
    const int xt = tpr >= nthr ? (int)threadIdx.x : (int)threadIdx.x % tpr;
    const int r0 = tpr >= nthr ? 0 : (int)threadIdx.x / tpr;
    const int xstride = tpr >= nthr ? nthr : tpr;
    const int nbj = ny / rows;
    const int k = blockIdx.x / nbj, j0 = (blockIdx.x % nbj) * rows;
    const bool hasup = !g.walls || k < nz - 1;
    const int ku = k == nz - 1 ? 0 : k + 1;
    const T idx = fpick<T>(g.idx, g.fidx), idy = fpick<T>(g.idy, g.fidy);
    const T idzk = Metric<T>::idz(g)[k];
    T m = T(0);
    for (int r = r0; r0 < rpp && r < rows; r += rpp) {
        const int j = j0 + r, jp = j == ny - 1 ? 0 : j + 1;
        const int oc = (k * ny + j) * nx, ojp = (k * ny + jp) * nx, oku = (ku * ny + j) * nx;
        for (int xv = xt; xv < tpr; xv += xstride) {
            const int i0 = xv * VW;
            const V a = *reinterpret_cast<const V *>(u + oc + i0);
            const V b = *reinterpret_cast<const V *>(v + oc + i0);
            const V bp = *reinterpret_cast<const V *>(v + ojp + i0);
            const V c = *reinterpret_cast<const V *>(w + oc + i0);
            V cu;
            if (hasup) cu = *reinterpret_cast<const V *>(w + oku + i0);
            const T an = u[oc + (i0 + VW == nx ? 0 : i0 + VW)];
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                const T uc = T(0.5) * (a.x[e] + (e == VW - 1 ? an : a.x[e + 1]));
                const T vc = T(0.5) * (b.x[e] + bp.x[e]);
                const T wku = hasup ? cu.x[e] : T(0);
                const T wc = T(0.5) * (c.x[e] + wku);
                m = fmax(m, fabs(uc) * idx + fabs(vc) * idy + fabs(wc) * idzk);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    __shared__ double wmax[32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = (double)m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = 0.0;
        for (int q = 0; q < (int)((blockDim.x + 31) >> 5); ++q) mm = fmax(mm, wmax[q]);
        atomicMax(&sc->speed_next, dbits(mm));
    }
}

// alpha and 1/c of the cyclic Toeplitz factorisation (tri.cuh, uni_solve)
// of (1 + 2r) I - r (E + E^-1)
__device__ void uni_factors(double r, double &alpha, double &cinv) {
    const double c = 0.5 * ((1.0 + 2.0 * r) + sqrt(1.0 + 4.0 * r));
    alpha = r / c;
    cinv = 1.0 / c;
}

// least n with alpha^n <= 2^-bits (0 <= alpha < 1), one more for the
// rounding of the logarithm; a large count where alpha is near 1
__device__ int decay_length(double alpha, int bits) {
    const double a = fabs(alpha);
    if (a == 0.0) return 1;
    const double l = -log2(a);
    if (!(l * (1 << 20) > bits)) return 1 << 20;
    return (int)ceil(bits / l) + 1;
}

// Three warps, so that the serial double-precision chains (each a division
// or square root at a time on GB300's narrow FP64 pipe) run side by side:
// every warp forms dt and beta (alpha dt_n, dt_n from dt or the CFL rule at
// substep 0, kept from substep 0 after it); warp 0 the x factors, warp 1 the
// y factors, warp 2 1/dt, the advection weights and the reset of the step's
// reductions.
// Lane 0 of each warp stores.
FSEI_D void k_scalars(StepScalars *sc, StepArgs a, int euler, double idx2, double idy2) {
    pdl_wait();
    pdl_trigger();
    const int wid = threadIdx.x >> 5;
    const bool lead = (threadIdx.x & 31) == 0;
    const unsigned long long spd = sc->speed_next;
    double dt_step = a.dt;
    if (a.substep > 0) {
        dt_step = sc->dt_step;   // the full step's dt, formed at substep 0
    } else if (a.cfl > 0.0) {
        const double s = bitsd(spd);
        dt_step = s > 0.0 ? a.cfl / s : a.dt;
    }
    const double dt = a.alpha * dt_step;
    const double beta = dt / (2.0 * a.re);
    __syncthreads();   // every warp has read speed_next before warp 2 resets it
    if (wid == 0) {
        double al, ci;
        uni_factors(beta * idx2, al, ci);
        if (lead) {
            sc->ax = al;
            sc->cix = ci;
            sc->fax = (float)al;
            sc->fcix = (float)ci;
            sc->ndecx_f = decay_length(al, 32);
            sc->ndecx_d = decay_length(al, 62);
        }
    } else if (wid == 1) {
        double al, ci;
        uni_factors(beta * idy2, al, ci);
        if (lead) {
            sc->ay = al;
            sc->ciy = ci;
            sc->fay = (float)al;
            sc->fciy = (float)ci;
        }
    } else if (lead) {
        const double invdt = 1.0 / dt;
        sc->speed_cur = spd;
        sc->speed_next = 0ull;
        sc->maxdiv = 0ull;
        sc->ke = 0.0;
        sc->flags = 0;
        sc->dt = dt;
        sc->dt_step = dt_step;
        sc->beta = beta;
        sc->gamma = euler ? 1.0 : a.gamma;
        sc->rho = euler ? 0.0 : a.rho;
        sc->invdt = invdt;
        sc->fdt = (float)dt;
        sc->fbeta = (float)beta;
        sc->fgamma = (float)sc->gamma;
        sc->frho = (float)sc->rho;
        sc->finvdt = (float)invdt;
    }
}

// Coefficients of the four sweep matrices, in double.  Row i of a line:
// a(i) x_{i-1} + b(i) x_i + c(i) x_{i+1}; a(0), c(n-1) are the periodic
// couplings of cyclic lines and 0 otherwise.
struct SweepCoef {
    int kind, n, nz, walls, pad;
    double beta, r;
    const double *idz, *ihc;
    FSEI_D double araw(int i) const {
        if (kind < 2) return -r;
        if (kind == 2) return -beta * ihc[i] * idz[i];
        if (walls) { const int k = i + 1; return -beta * idz[k - 1] * ihc[k]; }
        const int kd = i == 0 ? nz - 1 : i - 1;
        return -beta * idz[kd] * ihc[i];
    }
    FSEI_D double craw(int i) const {
        if (kind < 2) return -r;
        if (kind == 2) return -beta * ihc[i + 1] * idz[i];
        const int k = walls ? i + 1 : i;
        return -beta * idz[k] * ihc[k];
    }
    // rows past `last` are the padding identity rows
    FSEI_D int last() const { return n - 1 - pad; }
    FSEI_D double b(int i) const { return i > last() ? 1.0 : 1.0 - araw(i) - craw(i); }
    FSEI_D double a(int i) const {
        return (kind >= 2 && walls && (i == 0 || i > last())) ? 0.0 : araw(i);
    }
    FSEI_D double c(int i) const { return (kind >= 2 && walls && i >= last()) ? 0.0 : craw(i); }
};

// one block per plan; thread p < P builds chunk p; thread 0 the reduced LU
template <typename T>
FSEI_D void k_plans(GridDev g, ZPlans<T> Z, const StepScalars *sc) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int kind = 2 + blockIdx.x;   // the z plans (x and y lines use uni_solve)
    const TriPlan<T> &pl = Z.plan[blockIdx.x];
    const TriPlanStore<T> &st = Z.store[blockIdx.x];
    const int n = pl.n, P = pl.P;
    double *sat = reinterpret_cast<double *>(smraw);
    double *sct = sat + n;
    double *lo = sct + n, *di = lo + 2 * P, *up = di + 2 * P;
    SweepCoef cf;
    cf.kind = kind;
    cf.n = n;
    cf.nz = g.nz;
    cf.walls = g.walls;
    cf.pad = pl.pad;
    cf.beta = sc->beta;
    cf.r = kind == 0 ? sc->beta * g.idx2 : sc->beta * g.idy2;
    cf.idz = g.idz;
    cf.ihc = g.ihc;
    const int p = threadIdx.x;
    if (p < P) {
        const int s0 = chunk_start(p, n, P), e0 = chunk_start(p + 1, n, P) - 1;
        for (int i = s0; i <= e0; ++i) {
            st.a[i] = T(cf.a(i));
            st.c[i] = T(cf.c(i));
        }
        int i = s0 + 1;
        double inv = 1.0 / cf.b(i);
        double at = cf.a(i) * inv, ct = cf.c(i) * inv;
        sat[i] = at; sct[i] = ct;
        st.inv[i] = T(inv); st.at[i] = T(at); st.ct[i] = T(ct);
        for (i = s0 + 2; i < e0; ++i) {
            const double ai = cf.a(i);
            inv = 1.0 / (cf.b(i) - ai * ct);
            at = -ai * at * inv;
            ct = cf.c(i) * inv;
            sat[i] = at; sct[i] = ct;
            st.inv[i] = T(inv); st.at[i] = T(at); st.ct[i] = T(ct);
        }
        double ah = sat[e0 - 1], ch = sct[e0 - 1];
        const double ahe = ah, che = ch;
        for (i = e0 - 2; i > s0; --i) {
            ah = sat[i] - sct[i] * ah;
            ch = -sct[i] * ch;
        }
        lo[2 * p] = cf.a(s0);
        di[2 * p] = cf.b(s0) - cf.c(s0) * ah;
        up[2 * p] = -cf.c(s0) * ch;
        lo[2 * p + 1] = -cf.a(e0) * ahe;
        di[2 * p + 1] = cf.b(e0) - cf.a(e0) * che;
        up[2 * p + 1] = cf.c(e0);
    }
    __syncthreads();
    if (pl.levels > 0) {
        // parallel cyclic reduction multipliers of the reduced system: one
        // thread per equation, levels separated by barriers (in place over
        // copies of lo, di, up kept after the LU arrays)
        const int m = 2 * P;
        double *L = up + 2 * P, *D = L + m, *U = D + m;
        const int i = threadIdx.x;
        if (i < m) { L[i] = lo[i]; D[i] = di[i]; U[i] = up[i]; }
        __syncthreads();
        for (int lev = 0; lev < pl.levels; ++lev) {
            const int sft = 1 << lev;
            double nL = 0.0, nD = 0.0, nU = 0.0;
            if (i < m) {
                const int im = i - sft, ip = i + sft;
                const bool hm = pl.cyclic || im >= 0, hp = pl.cyclic || ip < m;
                const int jm = (im + m) & (m - 1), jp = ip & (m - 1);
                const double k1 = hm ? -L[i] / D[jm] : 0.0;
                const double k2 = hp ? -U[i] / D[jp] : 0.0;
                nD = D[i] + (hm ? k1 * U[jm] : 0.0) + (hp ? k2 * L[jp] : 0.0);
                nL = hm ? k1 * L[jm] : 0.0;
                nU = hp ? k2 * U[jp] : 0.0;
                st.pk1[lev * m + i] = T(k1);
                st.pk2[lev * m + i] = T(k2);
            }
            __syncthreads();
            if (i < m) { L[i] = nL; D[i] = nD; U[i] = nU; }
            __syncthreads();
        }
        // after the last level a cyclic equation couples only to itself
        if (i < m) st.pdinv[i] = T(1.0 / (D[i] + (pl.cyclic ? L[i] + U[i] : 0.0)));
    }
    __syncthreads();
    // Thomas factors of the reduced system: only needed without PCR
    if (threadIdx.x == 0 && pl.levels == 0) {
        const int m = 2 * P;
        const double g0 = -di[0];
        const double lo0 = lo[0], upm = up[m - 1];
        if (pl.cyclic) {
            di[0] -= g0;
            di[m - 1] -= upm * lo0 / g0;
        }
        double inv = 1.0 / di[0];
        double cp = up[0] * inv;
        st.rlo[0] = T(lo[0]); st.rinv[0] = T(inv); st.rcp[0] = T(cp);
        di[0] = inv; up[0] = cp;
        for (int j = 1; j < m; ++j) {
            inv = 1.0 / (di[j] - lo[j] * cp);
            cp = up[j] * inv;
            st.rlo[j] = T(lo[j]); st.rinv[j] = T(inv); st.rcp[j] = T(cp);
            di[j] = inv; up[j] = cp;
        }
        if (pl.cyclic) {
            // z = T^-1 (g0, 0, ..., 0, upm); stored in lo[] after use
            double z = g0 * di[0];
            lo[0] = z;
            for (int j = 1; j < m; ++j) {
                const double uj = (j == m - 1) ? upm : 0.0;
                z = di[j] * (uj - lo[j] * z);
                lo[j] = z;
            }
            for (int j = m - 2; j >= 0; --j) {
                z = lo[j] - up[j] * z;
                lo[j] = z;
            }
            const double vl = lo0 / g0;
            for (int j = 0; j < m; ++j) st.rz[j] = T(lo[j]);
            st.rsc[0] = T(vl);
            st.rsc[1] = T(1.0 / (1.0 + lo[0] + vl * lo[m - 1]));
        }
    }
}

// Stencil values around one point (i, j, k) read by the divergence-form
// advection, the Laplacian and the pressure gradient: u, v, w, p at the
// point and at its neighbours (ip/im: i +- 1, jp/jm: j +- 1, kp/km and
// ku/kd: k +- 1; a neighbour beyond a wall is 0).
template <typename T> struct Stencil {
    T u0, uip, uim, ujp, ujm, ukp, ukm, u_ip_jm, u_ip_kd;
    T v0, vip, vim, vjp, vjm, vkp, vkm, v_im_jp, v_jp_kd;
    T w0, wip, wim, wjp, wjm, wku, wkd, w_im_ku, w_jm_ku;
    T p0, pim, pjm, pkd;
};


// H^n = -div(uu)^n at the u, v and w points of cell (i, j, k) (products of
// two-point averages at the cell centres and edges, differenced) and RHS =
// dt [gamma H^n + rho H^{n-1} + Re^-1 L u^n - G p^n + f] (Eq. 3).  On the
// bottom wall face (wall_face) H_w and RHS_w are 0.
// the explicit extra term of F (if any) added to H and, with this step's
// weight dt gamma, to the right-hand side (0 on the bottom wall face)
template <typename T>
FSEI_D void add_extra_h(const Fields<T> &F, size_t c0, const RhsCoef<T> &c, T &Hu, T &Hv, T &Hw,
                        T &ru, T &rv, T &rw) {
    if (!F.hx) return;
    const T a = F.hx[c0], b = F.hy[c0], e = c.wall_face ? T(0) : F.hz[c0];
    const T dg = c.dt * c.gam;
    Hu += a;
    Hv += b;
    Hw += e;
    ru += dg * a;
    rv += dg * b;
    rw += dg * e;
}

template <typename T>
FSEI_D void rhs_point(const Stencil<T> &s, const RhsCoef<T> &c, T hu1, T hv1, T hw1, T fx, T fy,
                      T fz, T &Hu, T &Hv, T &Hw, T &ru, T &rv, T &rw) {
    const T h = T(0.5), z0 = T(0);
    // cross fluxes at the cell edges
    const T e_xy = (h * (s.v0 + s.vim)) * (h * (s.u0 + s.ujm));              // (x_i, y_j)
    const T e_xy_jp = (h * (s.vjp + s.v_im_jp)) * (h * (s.ujp + s.u0));      // (x_i, y_j+1)
    const T e_xy_ip = (h * (s.vip + s.v0)) * (h * (s.uip + s.u_ip_jm));      // (x_i+1, y_j)
    const T e_xz = c.hasdn ? (h * (s.w0 + s.wim)) * (h * (s.u0 + s.ukm)) : z0;
    const T e_xz_kp = c.hasup ? (h * (s.wku + s.w_im_ku)) * (h * (s.ukp + s.u0)) : z0;
    const T e_xz_ip = c.hasdn ? (h * (s.wip + s.w0)) * (h * (s.uip + s.u_ip_kd)) : z0;
    const T e_yz = c.hasdn ? (h * (s.w0 + s.wjm)) * (h * (s.v0 + s.vkm)) : z0;
    const T e_yz_kp = c.hasup ? (h * (s.wku + s.w_jm_ku)) * (h * (s.vkp + s.v0)) : z0;
    const T e_yz_jp = c.hasdn ? (h * (s.wjp + s.w0)) * (h * (s.vjp + s.v_jp_kd)) : z0;

    const T ucp = h * (s.u0 + s.uip), ucm = h * (s.uim + s.u0);
    Hu = -((ucp * ucp - ucm * ucm) * c.idx + (e_xy_jp - e_xy) * c.idy +
           (e_xz_kp - e_xz) * c.idzk);
    const T vcp = h * (s.v0 + s.vjp), vcm = h * (s.vjm + s.v0);
    Hv = -((e_xy_ip - e_xy) * c.idx + (vcp * vcp - vcm * vcm) * c.idy +
           (e_yz_kp - e_yz) * c.idzk);
    Hw = z0;
    if (!c.wall_face) {
        const T wcp = h * (s.w0 + s.wku), wcm = h * (s.wkd + s.w0);
        Hw = -((e_xz_ip - e_xz) * c.idx + (e_yz_jp - e_yz) * c.idy +
               (wcp * wcp - wcm * wcm) * c.ihck);
    }
    const T Lu = (s.uip - T(2) * s.u0 + s.uim) * c.idx2 + (s.ujp - T(2) * s.u0 + s.ujm) * c.idy2 +
                 ((s.ukp - s.u0) * c.ihcu - (s.u0 - s.ukm) * c.ihck) * c.idzk;
    const T Lv = (s.vip - T(2) * s.v0 + s.vim) * c.idx2 + (s.vjp - T(2) * s.v0 + s.vjm) * c.idy2 +
                 ((s.vkp - s.v0) * c.ihcu - (s.v0 - s.vkm) * c.ihck) * c.idzk;
    ru = c.dt * (c.gam * Hu + c.rho * hu1 + c.inv_re * Lu - (s.p0 - s.pim) * c.idx + fx + c.fc0);
    rv = c.dt * (c.gam * Hv + c.rho * hv1 + c.inv_re * Lv - (s.p0 - s.pjm) * c.idy + fy + c.fc1);
    rw = z0;
    if (!c.wall_face) {
        const T Lw = (s.wip - T(2) * s.w0 + s.wim) * c.idx2 +
                     (s.wjp - T(2) * s.w0 + s.wjm) * c.idy2 +
                     ((s.wku - s.w0) * c.idzk - (s.w0 - s.wkd) * c.idzd) * c.ihck;
        rw = c.dt * (c.gam * Hw + c.rho * hw1 + c.inv_re * Lw - (s.p0 - s.pkd) * c.ihck + fz +
                     c.fc2);
    }
}


// (I - beta L_x)^-1 along the nl = 3 ry right-hand-side lines of a block,
// held in sd[i * es + line] (line = component * ry + row), then stored as
// q0, q1, q2 rows j0 .. j0+ry-1 of plane k.  Thread t < nl P owns chunk
// t / nl of line t % nl in registers (uni_solve).  Every thread calls it.
template <typename T, int L>
FSEI_D void x_solve_store(T *sd, int es, int ry, int P, int nx, int ny, int k, int j0,
                          const StepScalars *sc, T *car, T *q0, T *q1, T *q2) {
    const int nl = 3 * ry;
    {
        const int t = threadIdx.x;
        const bool active = t < nl * P;
        const int p = active ? t / nl : 0, l = active ? t - p * nl : 0;
        const int s0 = chunk_start(p, nx, P);
        const int len = active ? chunk_start(p + 1, nx, P) - s0 : 0;
        T d[L];
#pragma unroll
        for (int i = 0; i < L; ++i)
            if (i < len) d[i] = sd[(s0 + i) * es + l];
        uni_solve<T, L>(d, len, active, l, p, nl, nx, P, fpick<T>(sc->ax, sc->fax),
                        fpick<T>(sc->cix, sc->fcix), car);
#pragma unroll
        for (int i = 0; i < L; ++i)
            if (i < len) sd[(s0 + i) * es + l] = d[i];
    }
    __syncthreads();
    for (int r = 0; r < ry; ++r) {
        const int o = (k * ny + j0 + r) * nx;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            q0[o + i] = sd[i * es + r];
            q1[o + i] = sd[i * es + ry + r];
            q2[o + i] = sd[i * es + 2 * ry + r];
        }
    }
}

// L: register chunk length of the x solve (>= nx / P).  Single precision
// keeps four blocks per SM for chunks of up to 16; longer chunks (nx > 256)
// take more registers.  General kernel (any nx): stencil values read from
// global memory; the tiled kernel below is used where it applies.
template <typename T, int L>
FSEI_D void
k_rhs_x(GridDev g, Fields<T> F, T *__restrict__ q0, T *__restrict__ q1, T *__restrict__ q2,
        const StepScalars *sc, int ry, int P, T fc0, T fc1, T fc2, T inv_re) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sd = reinterpret_cast<T *>(smraw);
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int nl = 3 * ry, es = nl | 1;
    T *car = sd + (size_t)nx * es;
    const int nby = ny / ry;
    const int k = blockIdx.x / nby, j0 = (blockIdx.x % nby) * ry;
    const RhsCoef<T> cf = rhs_coef<T>(g, sc, k, fc0, fc1, fc2, inv_re);
    const bool hasdn = cf.hasdn, hasup = cf.hasup;
    const int kd = k == 0 ? nz - 1 : k - 1, ku = k == nz - 1 ? 0 : k + 1;
    const T z0 = T(0);
    const T *__restrict__ u = F.u;
    const T *__restrict__ v = F.v;
    const T *__restrict__ w = F.w;
    const T *__restrict__ p = F.p;

    // 32-bit row offsets formed once per row (a field holds < 2^31 values);
    // the loads add them to the field base pointers (no wide multiplies)
    for (int r = 0; r < ry; ++r) {
      const int j = j0 + r;
      const int jp = j == ny - 1 ? 0 : j + 1, jm = j == 0 ? ny - 1 : j - 1;
      const int oc = (k * ny + j) * nx, ojp = (k * ny + jp) * nx, ojm = (k * ny + jm) * nx,
                oku = (ku * ny + j) * nx, okd = (kd * ny + j) * nx, ojpkd = (kd * ny + jp) * nx,
                ojmku = (ku * ny + jm) * nx;
      for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int ip = i == nx - 1 ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
        const int c0 = oc + i;
        Stencil<T> s;
        s.u0 = u[c0]; s.uip = u[oc + ip]; s.uim = u[oc + im];
        s.ujp = u[ojp + i]; s.ujm = u[ojm + i];
        s.ukp = hasup ? u[oku + i] : z0;
        s.ukm = hasdn ? u[okd + i] : z0;
        s.u_ip_jm = u[ojm + ip];
        s.u_ip_kd = hasdn ? u[okd + ip] : z0;
        s.v0 = v[c0]; s.vip = v[oc + ip]; s.vim = v[oc + im];
        s.vjp = v[ojp + i]; s.vjm = v[ojm + i];
        s.vkp = hasup ? v[oku + i] : z0;
        s.vkm = hasdn ? v[okd + i] : z0;
        s.v_im_jp = v[ojp + im];
        s.v_jp_kd = hasdn ? v[ojpkd + i] : z0;
        // w at the bottom wall face is stored as 0
        s.w0 = w[c0]; s.wip = w[oc + ip]; s.wim = w[oc + im];
        s.wjp = w[ojp + i]; s.wjm = w[ojm + i];
        s.wku = hasup ? w[oku + i] : z0;
        s.wkd = hasdn ? w[okd + i] : z0;
        s.w_im_ku = hasup ? w[oku + im] : z0;
        s.w_jm_ku = hasup ? w[ojmku + i] : z0;
        s.p0 = p[c0]; s.pim = p[oc + im]; s.pjm = p[ojm + i];
        s.pkd = hasdn ? p[okd + i] : z0;
        const T fx = F.fx ? F.fx[c0] : z0, fy = F.fy ? F.fy[c0] : z0;
        const T fz = (F.fz && !cf.wall_face) ? F.fz[c0] : z0;
        T Hu, Hv, Hw, ru, rv, rw;
        rhs_point(s, cf, F.hu[c0], F.hv[c0], F.hw[c0], fx, fy, fz, Hu, Hv, Hw, ru, rv, rw);
        add_extra_h(F, c0, cf, Hu, Hv, Hw, ru, rv, rw);
        F.hu[c0] = Hu;
        F.hv[c0] = Hv;
        F.hw[c0] = Hw;
        sd[i * es + r] = ru;
        sd[i * es + ry + r] = rv;
        sd[i * es + 2 * ry + r] = rw;
      }
    }
    __syncthreads();
    x_solve_store<T, L>(sd, es, ry, P, nx, ny, k, j0, sc, car, q0, q1, q2);
}

// Shared-memory rows of the tiled right-hand side for a block of RY rows
// j0 .. j0+RY-1 of plane k, by group (first row index; rows in y order):
//   plane k:   u, v, w rows j0-1 .. j0+RY; p rows j0-1 .. j0+RY-1;
//              H^{n-1} (hu, hv, hw) rows j0 .. j0+RY-1
//   plane k+1: u, v rows j0 .. j0+RY-1; w rows j0-1 .. j0+RY-1
//   plane k-1: u, w, p rows j0 .. j0+RY-1; v rows j0 .. j0+RY
// j wraps periodically; k +- 1 wraps when z is periodic and is absent (not
// copied, read as 0) beyond a wall.  14 RY + 9 rows in all.
struct TileRows {
    int u, v, w, p, hu, hv, hw, uu, vu, wu, ud, wd, pd, vd, total;
    FSEI_HD explicit TileRows(int RY) {
        int r = 0;
        u = r; r += RY + 2;
        v = r; r += RY + 2;
        w = r; r += RY + 2;
        p = r; r += RY + 1;
        hu = r; r += RY;
        hv = r; r += RY;
        hw = r; r += RY;
        uu = r; r += RY;
        vu = r; r += RY;
        wu = r; r += RY + 1;
        ud = r; r += RY;
        wd = r; r += RY;
        pd = r; r += RY;
        vd = r; r += RY + 1;
        total = r;
    }
};
constexpr int kTileRowsMax = 14 * 4 + 9;

// Element offset of a staged row's first value (16 bytes: the left x halo
// sits just before it) and the row stride: nx values plus one 16-byte slot
// on each side.
template <typename T> FSEI_HD int tile_xo() { return 16 / (int)sizeof(T); }
template <typename T> FSEI_HD int tile_rsz(int nx) { return nx + 2 * tile_xo<T>(); }

// Global row (field, plane kk, row jj) feeding staged row r, or NULL for a
// plane beyond a wall.
template <typename T>
FSEI_D const T *tile_source(const TileRows &tr, int RY, int r, const Fields<T> &F, int nx, int ny,
                            int k, int ku, int kd, bool hasup, bool hasdn, int j0) {
    const T *f;
    int kk, jrel;
    if (r < tr.v) { f = F.u; kk = k; jrel = r - tr.u - 1; }
    else if (r < tr.w) { f = F.v; kk = k; jrel = r - tr.v - 1; }
    else if (r < tr.p) { f = F.w; kk = k; jrel = r - tr.w - 1; }
    else if (r < tr.hu) { f = F.p; kk = k; jrel = r - tr.p - 1; }
    else if (r < tr.hv) { f = F.hu; kk = k; jrel = r - tr.hu; }
    else if (r < tr.hw) { f = F.hv; kk = k; jrel = r - tr.hv; }
    else if (r < tr.uu) { f = F.hw; kk = k; jrel = r - tr.hw; }
    else if (r < tr.vu) { f = hasup ? F.u : nullptr; kk = ku; jrel = r - tr.uu; }
    else if (r < tr.wu) { f = hasup ? F.v : nullptr; kk = ku; jrel = r - tr.vu; }
    else if (r < tr.ud) { f = hasup ? F.w : nullptr; kk = ku; jrel = r - tr.wu - 1; }
    else if (r < tr.wd) { f = hasdn ? F.u : nullptr; kk = kd; jrel = r - tr.ud; }
    else if (r < tr.pd) { f = hasdn ? F.w : nullptr; kk = kd; jrel = r - tr.wd; }
    else if (r < tr.vd) { f = hasdn ? F.p : nullptr; kk = kd; jrel = r - tr.pd; }
    else { f = hasdn ? F.v : nullptr; kk = kd; jrel = r - tr.vd; }
    if (!f) return nullptr;
    int j = j0 + jrel;
    if (j < 0) j += ny;
    if (j >= ny) j -= ny;
    return f + (kk * ny + j) * nx;
}

// Tiled right-hand side + x sweep: every stencil row of the block is
// staged in shared memory with 16-byte asynchronous copies (all in flight
// together), each staged row padded with its periodic x neighbours, so the
// point formula reads shared memory only.  Needs nx * sizeof(T) % 16 == 0.
// Same arithmetic, in the same order, as k_rhs_x.
template <typename T, int L, int RY>
FSEI_D void
k_rhs_x_tile(GridDev g, Fields<T> F, T *__restrict__ q0, T *__restrict__ q1,
             T *__restrict__ q2, const StepScalars *sc, int P, T fc0, T fc1, T fc2, T inv_re) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ const T *rowsrc[kTileRowsMax];
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const TileRows tr(RY);
    const int xo = tile_xo<T>(), rsz = tile_rsz<T>(nx);
    T *S = reinterpret_cast<T *>(smraw);
    const int nl = 3 * RY, es = nl | 1;
    T *sd = S + (size_t)tr.total * rsz;
    T *car = sd + (size_t)nx * es;
    const int nby = ny / RY;
    const int k = blockIdx.x / nby, j0 = (blockIdx.x % nby) * RY;
    const RhsCoef<T> cf = rhs_coef<T>(g, sc, k, fc0, fc1, fc2, inv_re);
    const int kd = k == 0 ? nz - 1 : k - 1, ku = k == nz - 1 ? 0 : k + 1;
    const int t = threadIdx.x;
    if (t < tr.total)
        rowsrc[t] = tile_source<T>(tr, RY, t, F, nx, ny, k, ku, kd, cf.hasup, cf.hasdn, j0);
    __syncthreads();
    {
        constexpr int VW = 16 / (int)sizeof(T);
        const int cpr = nx / VW;
        const int total = tr.total * cpr;
        for (int e = t; e < total; e += blockDim.x) {
            const int r = ddiv(e, cpr), c = e - r * cpr;
            const T *src = rowsrc[r];
            if (src) cp_async16(S + r * rsz + xo + c * VW, src + c * VW);
        }
        // periodic x neighbours of every row (plain loads, issued after the
        // asynchronous copies)
        for (int e = t; e < 2 * tr.total; e += blockDim.x) {
            const int r = e >> 1;
            const T *src = rowsrc[r];
            if (src) {
                if (e & 1) S[r * rsz + xo + nx] = src[0];
                else S[r * rsz + xo - 1] = src[nx - 1];
            }
        }
        cp_async_wait_all();
    }
    __syncthreads();
    const T z0 = T(0);
    const bool hasdn = cf.hasdn, hasup = cf.hasup;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const T *Uk = S + (tr.u + 1 + r) * rsz + xo, *Ujm = Uk - rsz, *Ujp = Uk + rsz;
        const T *Vk = S + (tr.v + 1 + r) * rsz + xo, *Vjm = Vk - rsz, *Vjp = Vk + rsz;
        const T *Wk = S + (tr.w + 1 + r) * rsz + xo, *Wjm = Wk - rsz, *Wjp = Wk + rsz;
        const T *Pk = S + (tr.p + 1 + r) * rsz + xo, *Pjm = Pk - rsz;
        const T *Hu1 = S + (tr.hu + r) * rsz + xo, *Hv1 = S + (tr.hv + r) * rsz + xo,
                *Hw1 = S + (tr.hw + r) * rsz + xo;
        const T *Uu = S + (tr.uu + r) * rsz + xo, *Vu = S + (tr.vu + r) * rsz + xo;
        const T *Wu = S + (tr.wu + 1 + r) * rsz + xo, *Wujm = Wu - rsz;
        const T *Ud = S + (tr.ud + r) * rsz + xo, *Wd = S + (tr.wd + r) * rsz + xo,
                *Pd = S + (tr.pd + r) * rsz + xo, *Vd = S + (tr.vd + r) * rsz + xo,
                *Vdjp = Vd + rsz;
        const int oc = (k * ny + j0 + r) * nx;
        for (int i = t; i < nx; i += blockDim.x) {
            const int c0 = oc + i;
            Stencil<T> s;
            s.u0 = Uk[i]; s.uip = Uk[i + 1]; s.uim = Uk[i - 1];
            s.ujp = Ujp[i]; s.ujm = Ujm[i];
            s.ukp = hasup ? Uu[i] : z0;
            s.ukm = hasdn ? Ud[i] : z0;
            s.u_ip_jm = Ujm[i + 1];
            s.u_ip_kd = hasdn ? Ud[i + 1] : z0;
            s.v0 = Vk[i]; s.vip = Vk[i + 1]; s.vim = Vk[i - 1];
            s.vjp = Vjp[i]; s.vjm = Vjm[i];
            s.vkp = hasup ? Vu[i] : z0;
            s.vkm = hasdn ? Vd[i] : z0;
            s.v_im_jp = Vjp[i - 1];
            s.v_jp_kd = hasdn ? Vdjp[i] : z0;
            s.w0 = Wk[i]; s.wip = Wk[i + 1]; s.wim = Wk[i - 1];
            s.wjp = Wjp[i]; s.wjm = Wjm[i];
            s.wku = hasup ? Wu[i] : z0;
            s.wkd = hasdn ? Wd[i] : z0;
            s.w_im_ku = hasup ? Wu[i - 1] : z0;
            s.w_jm_ku = hasup ? Wujm[i] : z0;
            s.p0 = Pk[i]; s.pim = Pk[i - 1]; s.pjm = Pjm[i];
            s.pkd = hasdn ? Pd[i] : z0;
            const T fx = F.fx ? F.fx[c0] : z0, fy = F.fy ? F.fy[c0] : z0;
            const T fz = (F.fz && !cf.wall_face) ? F.fz[c0] : z0;
            T Hu, Hv, Hw, ru, rv, rw;
            rhs_point(s, cf, Hu1[i], Hv1[i], Hw1[i], fx, fy, fz, Hu, Hv, Hw, ru, rv, rw);
            add_extra_h(F, c0, cf, Hu, Hv, Hw, ru, rv, rw);
            F.hu[c0] = Hu;
            F.hv[c0] = Hv;
            F.hw[c0] = Hw;
            sd[i * es + r] = ru;
            sd[i * es + RY + r] = rv;
            sd[i * es + 2 * RY + r] = rw;
        }
    }
    __syncthreads();
    x_solve_store<T, L>(sd, es, RY, P, nx, ny, k, j0, sc, car, q0, q1, q2);
}

// Row-resident right-hand side + x sweep reading its stencil rows straight
// from global memory: the LPR lanes of a warp segment (or of LPR / 32
// warps) own one x row (j, k), lane r cells CPL r .. CPL r + CPL - 1, read
// as 16-byte vectors or one 8-byte vector (neighbour rows are served by the
// caches).  Needs nx = LPR CPL, CPL values spanning 8 bytes or a multiple of
// 16, ny a multiple of rpb.
template <typename T, int CPL, int LPR>
FSEI_D void
k_rhs_x_row(GridDev g, Fields<T> F, T *__restrict__ q0, T *__restrict__ q1,
            T *__restrict__ q2, const StepScalars *sc, int rpb, T fc0, T fc1, T fc2, T inv_re) {
    // carries of the line solve: 2 x 3 values per thread (lines longer
    // than a warp; per warp on the exact scan)
    __shared__ T xs[LPR > 32 ? 2 * 3 * (LPR > 128 ? LPR : 128) : 1];
    pdl_wait();
    pdl_trigger();
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int nby = ny / rpb;
    const int k = blockIdx.x / nby;
    const int j = (blockIdx.x % nby) * rpb + (int)threadIdx.x / LPR;
    const int i0 = ((int)threadIdx.x & (LPR - 1)) * CPL;
    const RhsCoef<T> cf = rhs_coef<T>(g, sc, k, fc0, fc1, fc2, inv_re);
    const int kd = k == 0 ? nz - 1 : k - 1, ku = k == nz - 1 ? 0 : k + 1;
    const int jp = j == ny - 1 ? 0 : j + 1, jm = j == 0 ? ny - 1 : j - 1;
    auto row = [&](const T *f, int kk, int jj) { return f + (kk * ny + jj) * nx; };
    RowSet<T> rs;
    rs.U = row(F.u, k, j); rs.Ujm = row(F.u, k, jm); rs.Ujp = row(F.u, k, jp);
    rs.V = row(F.v, k, j); rs.Vjm = row(F.v, k, jm); rs.Vjp = row(F.v, k, jp);
    rs.W = row(F.w, k, j); rs.Wjm = row(F.w, k, jm); rs.Wjp = row(F.w, k, jp);
    rs.P = row(F.p, k, j); rs.Pjm = row(F.p, k, jm);
    rs.Uu = row(F.u, ku, j); rs.Vu = row(F.v, ku, j); rs.Wu = row(F.w, ku, j);
    rs.Wujm = row(F.w, ku, jm);
    rs.Ud = row(F.u, kd, j); rs.Vd = row(F.v, kd, j); rs.Vdjp = row(F.v, kd, jp);
    rs.Wd = row(F.w, kd, j); rs.Pd = row(F.p, kd, j);
    rs.H1u = row(F.hu, k, j); rs.H1v = row(F.hv, k, j); rs.H1w = row(F.hw, k, j);
    rhs_row_body<T, CPL, LPR>(g, F, rs, q0, q1, q2, sc, cf, (k * ny + j) * nx, i0, xs);
}

}  // namespace

// the kernels with their launch bounds
template <typename T> constexpr Kernel<k_speed<T>, 256, 0> K_speed{};
template <typename T> constexpr Kernel<k_speed_vec<T>, 128, 0> K_speed_vec{};
constexpr Kernel<k_scalars, 96, 0> K_scalars{};
template <typename T> constexpr Kernel<k_plans<T>, 128, 0> K_plans{};
template <typename T, int L>
constexpr Kernel<k_rhs_x<T, L>, 256, (L <= 16 ? (sizeof(T) == 4 ? 4 : 2) : (L <= 32 ? 2 : 1))>
    K_rhs_x{};
template <typename T, int L, int RY>
constexpr Kernel<k_rhs_x_tile<T, L, RY>, 256,
                 (sizeof(T) == 4 ? (L <= 16 ? 4 : (L <= 32 ? 3 : 2)) : (L <= 16 ? 2 : 1))>
    K_rhs_x_tile{};
template <typename T, int CPL, int LPR>
constexpr Kernel<k_rhs_x_row<T, CPL, LPR>, (LPR > 128 ? LPR : 128), 0> K_rhs_x_row{};

// ------------------------------------------------------------- launchers --
void uni_geometry(int n, int nl, int maxthr, int &P, int &chunk) {
    P = 1;
    while (P < 32 && nl * 2 * P <= maxthr) P *= 2;
    chunk = (n + P - 1) / P;
}

template <typename T> size_t smem_rhs_x(const GridDev &g, const Work<T> &W) {
    const int nl = 3 * W.ry, es = nl | 1;
    return sizeof(T) * ((size_t)g.nx * es + 2 * (size_t)nl * W.px);
}

template <typename T> void launch_speed(const GridDev &g, const T *u, const T *v, const T *w,
                                        StepScalars *sc, cudaStream_t st) {
    constexpr int VW = 16 / (int)sizeof(T);
    if (g.nx % VW == 0) {
        // 128 threads, about four row passes per thread
        const int tpr = g.nx / VW;
        const int rpp = tpr >= 128 ? 1 : 128 / tpr;
        int rows = 1;
        for (int r = 4 * rpp; r >= 1; --r)
            if (g.ny % r == 0) { rows = r; break; }
        K_speed_vec<T>.launch(false, dim3(g.nz * (g.ny / rows)), dim3(128), 0, st, g, u, v, w, sc, rows);
        return;
    }
    int rows = 1;
    for (int r = 8; r >= 1; r /= 2)
        if (g.ny % r == 0) { rows = r; break; }
    const int threads = g.nx >= 256 ? 256 : ((g.nx + 31) / 32) * 32;
    K_speed<T>.launch(false, dim3(g.nz * (g.ny / rows)), dim3(threads), 0, st, g, u, v, w, sc, rows);
}

void launch_step_scalars(const GridDev &g, StepScalars *sc, const StepArgs &a, int euler,
                         cudaStream_t st, bool pdl) {
    K_scalars.launch(pdl, dim3(1), dim3(96), 0, st, sc, a, euler, g.idx2, g.idy2);
}

template <typename T> void launch_step_plans(const GridDev &g, Work<T> &W, const StepScalars *sc,
                                             cudaStream_t st) {
    int maxn = 0, maxp = 0;
    for (int q = 2; q < 4; ++q) {
        if (W.plan[q].n > maxn) maxn = W.plan[q].n;
        if (W.plan[q].P > maxp) maxp = W.plan[q].P;
    }
    const size_t sm = sizeof(double) * (2 * (size_t)maxn + 12 * (size_t)maxp);
    int thr = ((2 * maxp + 31) / 32) * 32;   // 2 P <= 64 threads
    ZPlans<T> Z;
    for (int q = 0; q < 2; ++q) {
        Z.plan[q] = W.plan[2 + q];
        Z.store[q] = W.store[2 + q];
    }
    K_plans<T>.launch(false, dim3(2), dim3(thr), sm, st, g, Z, sc);
}

template <typename T> void launch_step_begin(const GridDev &g, Work<T> &W, StepScalars *sc,
                                             const StepArgs &a, int euler, cudaStream_t st) {
    launch_step_scalars(g, sc, a, euler, st);
    launch_step_plans<T>(g, W, sc, st);
}

template <typename T, int L>
void rhs_x_L(const GridDev &g, const Fields<T> &F, Work<T> &W, const StepScalars *sc,
             const StepArgs &a, cudaStream_t st) {
    const int nl = 3 * W.ry;
    int threads = ((nl * W.px + 31) / 32) * 32;
    // the right-hand-side phase strides over x: a block as wide as a row (up
    // to the 256-thread bound) avoids a mostly idle second pass per row
    const int row_threads = g.nx < 256 ? ((g.nx + 31) / 32) * 32 : 256;
    if (threads < row_threads) threads = row_threads;
    const int blocks = g.nz * (g.ny / W.ry);
    K_rhs_x<T, L>.launch(false, dim3(blocks), dim3(threads), smem_rhs_x(g, W), st, g, F, W.q0,
                         W.q1, W.q2, sc, W.ry, W.px, T(a.fconst[0]), T(a.fconst[1]),
                         T(a.fconst[2]), T(1.0 / a.re));
}

// Geometry of the tiled right-hand side: RY rows per block (2, else 1),
// P chunks per x line (the largest power of two <= 32 with 3 RY P <= 256
// threads and chunks of at least two unknowns), its shared memory; false
// where it does not apply (rows not 16-byte multiples, or too large for
// shared memory).
template <typename T> bool rhs_tile_geometry(const GridDev &g, int &RY, int &P, size_t &smem) {
    if ((g.nx * (int)sizeof(T)) % 16 != 0) return false;
    const size_t lim = (size_t)smem_optin() - 1024;
    for (RY = 2; RY >= 1; --RY) {
        if (g.ny % RY) continue;
        const int nl = 3 * RY, es = nl | 1;
        P = 1;
        while (P < 32 && nl * (2 * P) <= 256 && g.nx / (2 * P) >= 2) P *= 2;
        const TileRows tr(RY);
        smem = sizeof(T) * ((size_t)tr.total * tile_rsz<T>(g.nx) + (size_t)g.nx * es +
                            2 * (size_t)nl * P);
        if (smem <= lim) return true;
    }
    return false;
}

template <typename T, int L, int RY>
void rhs_tile_L(const GridDev &g, const Fields<T> &F, Work<T> &W, const StepScalars *sc,
                const StepArgs &a, int P, size_t smem, cudaStream_t st) {
    K_rhs_x_tile<T, L, RY>.launch(false, dim3(g.nz * (g.ny / RY)), dim3(256), smem, st, g, F,
                                  W.q0, W.q1, W.q2, sc, P, T(a.fconst[0]), T(a.fconst[1]),
                                  T(a.fconst[2]), T(1.0 / a.re));
}

template <typename T, int RY>
void rhs_tile_ry(const GridDev &g, const Fields<T> &F, Work<T> &W, const StepScalars *sc,
                 const StepArgs &a, int P, size_t smem, cudaStream_t st) {
    const int chunk = (g.nx + P - 1) / P;
    if (chunk <= 8) rhs_tile_L<T, 8, RY>(g, F, W, sc, a, P, smem, st);
    else if (chunk <= 16) rhs_tile_L<T, 16, RY>(g, F, W, sc, a, P, smem, st);
    else if (chunk <= 32) rhs_tile_L<T, 32, RY>(g, F, W, sc, a, P, smem, st);
    else rhs_tile_L<T, 64, RY>(g, F, W, sc, a, P, smem, st);
}

// Geometry of the row-resident right-hand side: CPL cells per lane, LPR =
// nx / CPL lanes per row (a power of two, 4 .. 256), rows per block rpb (a
// power of two dividing ny, the block of rpb LPR >= 32 threads at most
// max(128, LPR)); false where it does not apply.
template <typename T>
bool rhs_row_geometry(const GridDev &g, int &cpl, int &lpr, int &rpb, int prefer) {
    // 4 cells per lane (2 doubles or 4 floats: fewer registers, more warps);
    // floats on rows wider than 256 cells take 8; rows of 3 x 2^m cells
    // take 24-byte lanes (6 floats, 3 doubles); `prefer` (4 or the 24-byte
    // count, or 2 or 8 in single precision, from the grid's autotuner)
    // overrides
    auto fits = [&](int c) {
        const int l = g.nx % c ? 0 : g.nx / c;
        return l >= 4 && l <= 256 && (l & (l - 1)) == 0;
    };
    const int c24 = sizeof(T) == 4 ? 6 : 3;
    cpl = (sizeof(T) == 4 && g.nx > 256) ? 8 : 4;
    if (!fits(cpl) && fits(c24)) cpl = c24;
    if (prefer == 4 || prefer == c24 || ((prefer == 8 || prefer == 2) && sizeof(T) == 4))
        cpl = prefer;
    if (!fits(cpl) || (cpl == c24 && (g.nx / cpl < 8 || g.nx / cpl > 128))) return false;
    lpr = g.nx / cpl;
    const int bmax = lpr > 128 ? lpr : 128;
    for (rpb = bmax / lpr; rpb >= 1; rpb /= 2)
        if (g.ny % rpb == 0 && rpb * lpr >= 32) return true;
    return false;
}

template <typename T, int CPL, int LPR>
void rhs_row_launch(const GridDev &g, const Fields<T> &F, Work<T> &W, const StepScalars *sc,
                    const StepArgs &a, int rpb, cudaStream_t st) {
    K_rhs_x_row<T, CPL, LPR>.launch(W.pdl != 0, dim3(g.nz * (g.ny / rpb)), dim3(rpb * LPR), 0,
                                    st, g, F, W.q0, W.q1, W.q2, sc, rpb, T(a.fconst[0]),
                                    T(a.fconst[1]), T(a.fconst[2]), T(1.0 / a.re));
}

template <typename T, int CPL>
bool rhs_row_dispatch(const GridDev &g, const Fields<T> &F, Work<T> &W, const StepScalars *sc,
                      const StepArgs &a, int lpr, int rpb, cudaStream_t st) {
    switch (lpr) {
    case 4: rhs_row_launch<T, CPL, 4>(g, F, W, sc, a, rpb, st); return true;
    case 8: rhs_row_launch<T, CPL, 8>(g, F, W, sc, a, rpb, st); return true;
    case 16: rhs_row_launch<T, CPL, 16>(g, F, W, sc, a, rpb, st); return true;
    case 32: rhs_row_launch<T, CPL, 32>(g, F, W, sc, a, rpb, st); return true;
    case 64: rhs_row_launch<T, CPL, 64>(g, F, W, sc, a, rpb, st); return true;
    case 128: rhs_row_launch<T, CPL, 128>(g, F, W, sc, a, rpb, st); return true;
    case 256: rhs_row_launch<T, CPL, 256>(g, F, W, sc, a, rpb, st); return true;
    default: return false;
    }
}

// 24-byte lanes (rows of 3 x 2^m cells): 8 to 128 lanes per row
template <typename T>
bool rhs_row_dispatch24(const GridDev &g, const Fields<T> &F, Work<T> &W, const StepScalars *sc,
                        const StepArgs &a, int lpr, int rpb, cudaStream_t st) {
    constexpr int C = sizeof(T) == 4 ? 6 : 3;
    switch (lpr) {
    case 8: rhs_row_launch<T, C, 8>(g, F, W, sc, a, rpb, st); return true;
    case 16: rhs_row_launch<T, C, 16>(g, F, W, sc, a, rpb, st); return true;
    case 32: rhs_row_launch<T, C, 32>(g, F, W, sc, a, rpb, st); return true;
    case 64: rhs_row_launch<T, C, 64>(g, F, W, sc, a, rpb, st); return true;
    case 128: rhs_row_launch<T, C, 128>(g, F, W, sc, a, rpb, st); return true;
    default: return false;
    }
}

template <typename T> void launch_rhs_x(const GridDev &g, const Fields<T> &F, Work<T> &W,
                                        const StepScalars *sc, const StepArgs &a, cudaStream_t st) {
    if (W.rhs_strip > 0 && launch_rhs_x_march<T>(g, F, W, sc, a, st)) return;
    int cpl = 0, lpr = 0, rpb = 0;
    if (rhs_row_geometry<T>(g, cpl, lpr, rpb, W.rhs_cpl) &&
        (cpl == 4   ? rhs_row_dispatch<T, 4>(g, F, W, sc, a, lpr, rpb, st)
         : cpl == 8 ? rhs_row_dispatch<T, sizeof(T) == 4 ? 8 : 4>(g, F, W, sc, a, lpr, rpb, st)
         : cpl == 2 ? rhs_row_dispatch<T, sizeof(T) == 4 ? 2 : 4>(g, F, W, sc, a, lpr, rpb, st)
                    : rhs_row_dispatch24<T>(g, F, W, sc, a, lpr, rpb, st)))
        return;
    int RY = 0, P = 0;
    size_t smem = 0;
    if (rhs_tile_geometry<T>(g, RY, P, smem)) {
        if (RY == 2) rhs_tile_ry<T, 2>(g, F, W, sc, a, P, smem, st);
        else rhs_tile_ry<T, 1>(g, F, W, sc, a, P, smem, st);
        return;
    }
    if (W.chunk_x <= 8) rhs_x_L<T, 8>(g, F, W, sc, a, st);
    else if (W.chunk_x <= 16) rhs_x_L<T, 16>(g, F, W, sc, a, st);
    else if (W.chunk_x <= 32) rhs_x_L<T, 32>(g, F, W, sc, a, st);
    else rhs_x_L<T, 64>(g, F, W, sc, a, st);
}

int rhs_cpl_candidates(const GridDev &g, int elem_size, int *out, int cap) {
    int n = 0;
    const int opts[5] = {4, 8, 2, 6, 3};
    for (int c : opts) {
        int cpl = 0, lpr = 0, rpb = 0;
        const bool ok = elem_size == 4 ? rhs_row_geometry<float>(g, cpl, lpr, rpb, c)
                                       : rhs_row_geometry<double>(g, cpl, lpr, rpb, c);
        if (ok && cpl == c && n < cap) out[n++] = c;
    }
    return n;
}

template <typename T> void set_smem_limits_sweep(const GridDev &g, const Work<T> &W) {
    // load every kernel of this file now: a kernel loaded lazily at its first
    // launch cannot be loaded inside a stream capture
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, K_speed<T>.solo());
    cudaFuncGetAttributes(&fa, K_speed_vec<T>.solo());
    cudaFuncGetAttributes(&fa, K_scalars.solo());
    cudaFuncGetAttributes(&fa, K_plans<T>.solo());
    (void)g;
    (void)W;
    raise_smem_limit(K_rhs_x<T, 8>.solo());
    raise_smem_limit(K_rhs_x<T, 16>.solo());
    raise_smem_limit(K_rhs_x<T, 32>.solo());
    raise_smem_limit(K_rhs_x<T, 64>.solo());
    raise_smem_limit(K_rhs_x_tile<T, 8, 1>.solo());
    raise_smem_limit(K_rhs_x_tile<T, 16, 1>.solo());
    raise_smem_limit(K_rhs_x_tile<T, 32, 1>.solo());
    raise_smem_limit(K_rhs_x_tile<T, 64, 1>.solo());
    raise_smem_limit(K_rhs_x_tile<T, 8, 2>.solo());
    raise_smem_limit(K_rhs_x_tile<T, 16, 2>.solo());
    raise_smem_limit(K_rhs_x_tile<T, 32, 2>.solo());
    raise_smem_limit(K_rhs_x_tile<T, 64, 2>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, 4, 4>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, 4, 8>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, 4, 16>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, 4, 32>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, 4, 64>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, 4, 128>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, 4, 256>.solo());
    constexpr int C = sizeof(T) == 4 ? 8 : 4;
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C, 4>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C, 8>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C, 16>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C, 32>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C, 64>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C, 128>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C, 256>.solo());
    constexpr int C2 = sizeof(T) == 4 ? 2 : 4;
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C2, 4>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C2, 8>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C2, 16>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C2, 32>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C2, 64>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C2, 128>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C2, 256>.solo());
    constexpr int C24 = sizeof(T) == 4 ? 6 : 3;
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C24, 8>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C24, 16>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C24, 32>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C24, 64>.solo());
    cudaFuncGetAttributes(&fa, K_rhs_x_row<T, C24, 128>.solo());
}

#define FSEI_INST(T)                                                                           \
    template size_t smem_rhs_x<T>(const GridDev &, const Work<T> &);                          \
    template void launch_speed<T>(const GridDev &, const T *, const T *, const T *,            \
                                  StepScalars *, cudaStream_t);                               \
    template void launch_step_begin<T>(const GridDev &, Work<T> &, StepScalars *,              \
                                       const StepArgs &, int, cudaStream_t);                  \
    template void launch_step_plans<T>(const GridDev &, Work<T> &, const StepScalars *,        \
                                       cudaStream_t);                                         \
    template void launch_rhs_x<T>(const GridDev &, const Fields<T> &, Work<T> &,               \
                                  const StepScalars *, const StepArgs &, cudaStream_t);       \
    template void set_smem_limits_sweep<T>(const GridDev &, const Work<T> &);                 \
    template bool rhs_row_geometry<T>(const GridDev &, int &, int &, int &, int);
FSEI_INST(float)
FSEI_INST(double)
#undef FSEI_INST

}  // namespace fsei
