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
#include "tri.cuh"

namespace fsei {

namespace {

// one block per group of rows (no integer division per element); per-cell
// speed in the field precision, the grid-wide maximum in double
template <typename T>
__global__ void __launch_bounds__(256)
k_speed(GridDev g, const T *__restrict__ u, const T *__restrict__ v, const T *__restrict__ w,
        StepScalars *sc, int rows) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int nbj = ny / rows;
    const int k = blockIdx.x / nbj, j0 = (blockIdx.x % nbj) * rows;
    const bool hasup = !g.walls || k < nz - 1;
    const int ku = k == nz - 1 ? 0 : k + 1;
    const T idx = T(g.idx), idy = T(g.idy), idzk = Metric<T>::idz(g)[k];
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

// alpha and 1/c of the cyclic Toeplitz factorisation (tri.cuh, uni_solve)
// of (1 + 2r) I - r (E + E^-1)
__device__ void uni_factors(double r, double &alpha, double &cinv) {
    const double c = 0.5 * ((1.0 + 2.0 * r) + sqrt(1.0 + 4.0 * r));
    alpha = r / c;
    cinv = 1.0 / c;
}

__global__ void k_scalars(StepScalars *sc, StepArgs a, int euler, double idx2, double idy2) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double dt = a.dt;
    if (a.cfl > 0.0) {
        const double s = bitsd(sc->speed_next);
        dt = s > 0.0 ? a.cfl / s : a.dt;
    }
    sc->speed_cur = sc->speed_next;
    sc->speed_next = 0ull;
    sc->maxdiv = 0ull;
    sc->ke = 0.0;
    sc->flags = 0;
    sc->dt = dt;
    sc->beta = dt / (2.0 * a.re);
    uni_factors(sc->beta * idx2, sc->ax, sc->cix);
    uni_factors(sc->beta * idy2, sc->ay, sc->ciy);
    sc->gamma = euler ? 1.0 : a.gamma;
    sc->rho = euler ? 0.0 : a.rho;
}

// Coefficients of the four sweep matrices, in double.  Row i of a line:
// a(i) x_{i-1} + b(i) x_i + c(i) x_{i+1}; a(0), c(n-1) are the periodic
// couplings of cyclic lines and 0 otherwise.
struct SweepCoef {
    int kind, n, nz, walls;
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
    FSEI_D double b(int i) const { return 1.0 - araw(i) - craw(i); }
    FSEI_D double a(int i) const { return (kind >= 2 && walls && i == 0) ? 0.0 : araw(i); }
    FSEI_D double c(int i) const { return (kind >= 2 && walls && i == n - 1) ? 0.0 : craw(i); }
};

// one block per plan; thread p < P builds chunk p; thread 0 the reduced LU
template <typename T>
__global__ void k_plans(GridDev g, Work<T> W, const StepScalars *sc) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int kind = 2 + blockIdx.x;   // the z plans (x and y lines use uni_solve)
    const TriPlan<T> &pl = W.plan[kind];
    const TriPlanStore<T> &st = W.store[kind];
    const int n = pl.n, P = pl.P;
    double *sat = reinterpret_cast<double *>(smraw);
    double *sct = sat + n;
    double *lo = sct + n, *di = lo + 2 * P, *up = di + 2 * P;
    SweepCoef cf;
    cf.kind = kind;
    cf.n = n;
    cf.nz = g.nz;
    cf.walls = g.walls;
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

// L: register chunk length of the x solve (>= nx / P).  Single precision
// keeps four blocks per SM for chunks of up to 16; longer chunks (nx > 256)
// take more registers.
template <typename T, int L>
__global__ void __launch_bounds__(256, L <= 16 ? (sizeof(T) == 4 ? 4 : 2) : (L <= 32 ? 2 : 1))
k_rhs_x(GridDev g, Fields<T> F, T *__restrict__ q0, T *__restrict__ q1, T *__restrict__ q2,
        const StepScalars *sc, int ry, int P, T fc0, T fc1, T fc2, T inv_re) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sd = reinterpret_cast<T *>(smraw);
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int nl = 3 * ry, es = nl | 1;
    T *car = sd + (size_t)nx * es;
    const int nby = ny / ry;
    const int k = blockIdx.x / nby, j0 = (blockIdx.x % nby) * ry;
    const T dt = T(sc->dt), gam = T(sc->gamma), rho = T(sc->rho);
    const T *idz = Metric<T>::idz(g), *ihc = Metric<T>::ihc(g);
    const T idx = T(g.idx), idy = T(g.idy), idx2 = T(g.idx2), idy2 = T(g.idy2);
    const bool walls = g.walls != 0;
    const bool hasdn = !walls || k > 0, hasup = !walls || k < nz - 1;
    const bool wall_face = walls && k == 0;
    const int kd = k == 0 ? nz - 1 : k - 1, ku = k == nz - 1 ? 0 : k + 1;
    const T idzk = idz[k], idzd = idz[kd], ihck = ihc[k], ihcu = ihc[k + 1];
    const T h = T(0.5), z0 = T(0);
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
        // u neighbourhood
        const T u0 = u[c0], uip = u[oc + ip], uim = u[oc + im];
        const T ujp = u[ojp + i], ujm = u[ojm + i];
        const T ukp = hasup ? u[oku + i] : z0;
        const T ukm = hasdn ? u[okd + i] : z0;
        const T u_ip_jm = u[ojm + ip];
        const T u_ip_kd = hasdn ? u[okd + ip] : z0;
        // v neighbourhood
        const T v0 = v[c0], vip = v[oc + ip], vim = v[oc + im];
        const T vjp = v[ojp + i], vjm = v[ojm + i];
        const T vkp = hasup ? v[oku + i] : z0;
        const T vkm = hasdn ? v[okd + i] : z0;
        const T v_im_jp = v[ojp + im];
        const T v_jp_kd = hasdn ? v[ojpkd + i] : z0;
        // w neighbourhood (w at the bottom wall face is stored as 0)
        const T w0 = w[c0], wip = w[oc + ip], wim = w[oc + im];
        const T wjp = w[ojp + i], wjm = w[ojm + i];
        const T wku = hasup ? w[oku + i] : z0;
        const T wkd = hasdn ? w[okd + i] : z0;
        const T w_im_ku = hasup ? w[oku + im] : z0;
        const T w_jm_ku = hasup ? w[ojmku + i] : z0;
        // p
        const T p0 = p[c0], pim = p[oc + im], pjm = p[ojm + i];
        const T pkd = hasdn ? p[okd + i] : z0;

        // cross fluxes at the cell edges
        const T e_xy = (h * (v0 + vim)) * (h * (u0 + ujm));          // (x_i, y_j)
        const T e_xy_jp = (h * (vjp + v_im_jp)) * (h * (ujp + u0));  // (x_i, y_j+1)
        const T e_xy_ip = (h * (vip + v0)) * (h * (uip + u_ip_jm));  // (x_i+1, y_j)
        const T e_xz = hasdn ? (h * (w0 + wim)) * (h * (u0 + ukm)) : z0;          // (x_i, z_k)
        const T e_xz_kp = hasup ? (h * (wku + w_im_ku)) * (h * (ukp + u0)) : z0;  // (x_i, z_k+1)
        const T e_xz_ip = hasdn ? (h * (wip + w0)) * (h * (uip + u_ip_kd)) : z0;  // (x_i+1, z_k)
        const T e_yz = hasdn ? (h * (w0 + wjm)) * (h * (v0 + vkm)) : z0;
        const T e_yz_kp = hasup ? (h * (wku + w_jm_ku)) * (h * (vkp + v0)) : z0;
        const T e_yz_jp = hasdn ? (h * (wjp + w0)) * (h * (vjp + v_jp_kd)) : z0;

        const T ucp = h * (u0 + uip), ucm = h * (uim + u0);
        const T Hu = -((ucp * ucp - ucm * ucm) * idx + (e_xy_jp - e_xy) * idy +
                       (e_xz_kp - e_xz) * idzk);
        const T vcp = h * (v0 + vjp), vcm = h * (vjm + v0);
        const T Hv = -((e_xy_ip - e_xy) * idx + (vcp * vcp - vcm * vcm) * idy +
                       (e_yz_kp - e_yz) * idzk);
        T Hw = z0;
        if (!wall_face) {
            const T wcp = h * (w0 + wku), wcm = h * (wkd + w0);
            Hw = -((e_xz_ip - e_xz) * idx + (e_yz_jp - e_yz) * idy + (wcp * wcp - wcm * wcm) * ihck);
        }
        const T Lu = (uip - T(2) * u0 + uim) * idx2 + (ujp - T(2) * u0 + ujm) * idy2 +
                     ((ukp - u0) * ihcu - (u0 - ukm) * ihck) * idzk;
        const T Lv = (vip - T(2) * v0 + vim) * idx2 + (vjp - T(2) * v0 + vjm) * idy2 +
                     ((vkp - v0) * ihcu - (v0 - vkm) * ihck) * idzk;
        const T fx = F.fx ? F.fx[c0] : z0, fy = F.fy ? F.fy[c0] : z0;
        const T ru = dt * (gam * Hu + rho * F.hu[c0] + inv_re * Lu - (p0 - pim) * idx + fx + fc0);
        const T rv = dt * (gam * Hv + rho * F.hv[c0] + inv_re * Lv - (p0 - pjm) * idy + fy + fc1);
        T rw = z0;
        if (!wall_face) {
            const T Lw = (wip - T(2) * w0 + wim) * idx2 + (wjp - T(2) * w0 + wjm) * idy2 +
                         ((wku - w0) * idzk - (w0 - wkd) * idzd) * ihck;
            const T fz = F.fz ? F.fz[c0] : z0;
            rw = dt * (gam * Hw + rho * F.hw[c0] + inv_re * Lw - (p0 - pkd) * ihck + fz + fc2);
        }
        F.hu[c0] = Hu;
        F.hv[c0] = Hv;
        F.hw[c0] = Hw;
        sd[i * es + r] = ru;
        sd[i * es + ry + r] = rv;
        sd[i * es + 2 * ry + r] = rw;
      }
    }
    __syncthreads();
    // (I - beta L_x)^-1 along the nl lines: thread t < nl P owns chunk
    // t / nl of line t % nl in registers
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
        uni_solve<T, L>(d, len, active, l, p, nl, nx, P, T(sc->ax), T(sc->cix), car);
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

}  // namespace

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
    int rows = 1;
    for (int r = 8; r >= 1; r /= 2)
        if (g.ny % r == 0) { rows = r; break; }
    const int threads = g.nx >= 256 ? 256 : ((g.nx + 31) / 32) * 32;
    k_speed<T><<<g.nz * (g.ny / rows), threads, 0, st>>>(g, u, v, w, sc, rows);
}

template <typename T> void launch_step_begin(const GridDev &g, Work<T> &W, StepScalars *sc,
                                             const StepArgs &a, int euler, cudaStream_t st) {
    k_scalars<<<1, 32, 0, st>>>(sc, a, euler, g.idx2, g.idy2);
    int maxn = 0, maxp = 0;
    for (int q = 2; q < 4; ++q) {
        if (W.plan[q].n > maxn) maxn = W.plan[q].n;
        if (W.plan[q].P > maxp) maxp = W.plan[q].P;
    }
    const size_t sm = sizeof(double) * (2 * (size_t)maxn + 12 * (size_t)maxp);
    int thr = ((2 * maxp + 31) / 32) * 32;
    k_plans<T><<<2, thr, sm, st>>>(g, W, sc);
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
    k_rhs_x<T, L><<<blocks, threads, smem_rhs_x(g, W), st>>>(
        g, F, W.q0, W.q1, W.q2, sc, W.ry, W.px, T(a.fconst[0]), T(a.fconst[1]), T(a.fconst[2]),
        T(1.0 / a.re));
}

template <typename T> void launch_rhs_x(const GridDev &g, const Fields<T> &F, Work<T> &W,
                                        const StepScalars *sc, const StepArgs &a, cudaStream_t st) {
    if (W.chunk_x <= 8) rhs_x_L<T, 8>(g, F, W, sc, a, st);
    else if (W.chunk_x <= 16) rhs_x_L<T, 16>(g, F, W, sc, a, st);
    else if (W.chunk_x <= 32) rhs_x_L<T, 32>(g, F, W, sc, a, st);
    else rhs_x_L<T, 64>(g, F, W, sc, a, st);
}

template <typename T> void set_smem_limits_sweep(const GridDev &g, const Work<T> &W) {
    // load every kernel of this file now: a kernel loaded lazily at its first
    // launch cannot be loaded inside a stream capture
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_speed<T>);
    cudaFuncGetAttributes(&fa, k_scalars);
    cudaFuncGetAttributes(&fa, k_plans<T>);
    (void)g;
    (void)W;
    raise_smem_limit(k_rhs_x<T, 8>);
    raise_smem_limit(k_rhs_x<T, 16>);
    raise_smem_limit(k_rhs_x<T, 32>);
    raise_smem_limit(k_rhs_x<T, 64>);
}

#define FSEI_INST(T)                                                                           \
    template size_t smem_rhs_x<T>(const GridDev &, const Work<T> &);                          \
    template void launch_speed<T>(const GridDev &, const T *, const T *, const T *,            \
                                  StepScalars *, cudaStream_t);                               \
    template void launch_step_begin<T>(const GridDev &, Work<T> &, StepScalars *,              \
                                       const StepArgs &, int, cudaStream_t);                  \
    template void launch_rhs_x<T>(const GridDev &, const Fields<T> &, Work<T> &,               \
                                  const StepScalars *, const StepArgs &, cudaStream_t);       \
    template void set_smem_limits_sweep<T>(const GridDev &, const Work<T> &);
FSEI_INST(float)
FSEI_INST(double)
#undef FSEI_INST

}  // namespace fsei
