// Right-hand side of one grid row and its x sweep, shared by the
// row-resident kernels (Sec. 2.1, Eq. 3: H^n = -div(uu)^n, RHS = dt[gamma
// H^n + rho H^{n-1} + Re^-1 L u^n - G p^n + f]; Sec. 3.1: the x factor
// (I - beta L_x) solved on the registers of the row's lanes).
#pragma once

#include "kernels.cuh"
#include "tri.cuh"

namespace fsei {
namespace {

// 16 bytes of consecutive values (4 floats or 2 doubles)
template <typename T> struct alignas(16) Vec16 {
    static constexpr int W = 16 / (int)sizeof(T);
    T v[W];
};

// Step and plane-k coefficients of the point formula.
template <typename T> struct RhsCoef {
    T dt, gam, rho, inv_re, idx, idy, idx2, idy2, idzk, idzd, ihck, ihcu, fc0, fc1, fc2;
    bool hasdn, hasup, wall_face;
};

template <typename T>
FSEI_D RhsCoef<T> rhs_coef(const GridDev &g, const StepScalars *sc, int k, T fc0, T fc1, T fc2,
                           T inv_re) {
    RhsCoef<T> c;
    const T *idz = Metric<T>::idz(g), *ihc = Metric<T>::ihc(g);
    const int nz = g.nz;
    const bool walls = g.walls != 0;
    const int kd = k == 0 ? nz - 1 : k - 1;
    c.dt = fpick<T>(sc->dt, sc->fdt);
    c.gam = fpick<T>(sc->gamma, sc->fgamma);
    c.rho = fpick<T>(sc->rho, sc->frho);
    c.inv_re = inv_re;
    c.idx = fpick<T>(g.idx, g.fidx);
    c.idy = fpick<T>(g.idy, g.fidy);
    c.idx2 = fpick<T>(g.idx2, g.fidx2);
    c.idy2 = fpick<T>(g.idy2, g.fidy2);
    c.idzk = idz[k];
    c.idzd = idz[kd];
    c.ihck = ihc[k];
    c.ihcu = ihc[k + 1];
    c.fc0 = fc0;
    c.fc1 = fc1;
    c.fc2 = fc2;
    c.hasdn = !walls || k > 0;
    c.hasup = !walls || k < nz - 1;
    c.wall_face = walls && k == 0;
    return c;
}

// Helpers of the row-resident right-hand side (k_rhs_x_row below): CPL
// consecutive values of a row as 16-byte vectors where the lane holds a
// multiple of 16 bytes, as 8-byte vectors otherwise (8 or 24 bytes), from and
// to global memory (neighbour rows are served by the caches).
template <typename T> struct alignas(8) Vec8 { T v[8 / sizeof(T)]; };
template <typename T, int CPL>
FSEI_D void ldrow(T (&a)[CPL], const T *p) {
    static_assert((CPL * sizeof(T)) % 8 == 0, "8-byte multiple per lane");
    if constexpr ((CPL * sizeof(T)) % 16 != 0) {
        constexpr int VW = 8 / (int)sizeof(T);
#pragma unroll
        for (int c = 0; c < CPL / VW; ++c) {
            const Vec8<T> v = *reinterpret_cast<const Vec8<T> *>(p + c * VW);
#pragma unroll
            for (int e = 0; e < VW; ++e) a[c * VW + e] = v.v[e];
        }
    } else {
        constexpr int VW = 16 / (int)sizeof(T);
#pragma unroll
        for (int c = 0; c < CPL / VW; ++c) {
            const Vec16<T> v = *reinterpret_cast<const Vec16<T> *>(p + c * VW);
#pragma unroll
            for (int e = 0; e < VW; ++e) a[c * VW + e] = v.v[e];
        }
    }
}
template <typename T, int CPL>
FSEI_D void strow(T *p, const T (&a)[CPL]) {
    if constexpr ((CPL * sizeof(T)) % 16 != 0) {
        constexpr int VW = 8 / (int)sizeof(T);
#pragma unroll
        for (int c = 0; c < CPL / VW; ++c) {
            Vec8<T> v;
#pragma unroll
            for (int e = 0; e < VW; ++e) v.v[e] = a[c * VW + e];
            *reinterpret_cast<Vec8<T> *>(p + c * VW) = v;
        }
    } else {
        constexpr int VW = 16 / (int)sizeof(T);
#pragma unroll
        for (int c = 0; c < CPL / VW; ++c) {
            Vec16<T> v;
#pragma unroll
            for (int e = 0; e < VW; ++e) v.v[e] = a[c * VW + e];
            *reinterpret_cast<Vec16<T> *>(p + c * VW) = v;
        }
    }
}
// value of the periodic x neighbour left (LEFT = 1) of this lane's first
// cell, or right of its last one: from the neighbouring lane of the line
// (mine: this lane's last / first value), or, where the line crosses a warp
// boundary, from the row in memory
template <typename T, int LPR, int LEFT>
FSEI_D T xnb(T mine, const T *row, int i0, int nx, int CPL) {
    constexpr int W = LPR < 32 ? LPR : 32;
    const int p = threadIdx.x & (W - 1);
    T v = __shfl_sync(0xffffffffu, mine, LEFT ? ((p - 1) & (W - 1)) : ((p + 1) & (W - 1)), W);
    if (LPR > 32) {
        if (LEFT && p == 0) v = row[i0 == 0 ? nx - 1 : i0 - 1];
        if (!LEFT && p == W - 1) v = row[i0 + CPL == nx ? 0 : i0 + CPL];
    }
    return v;
}

// The rows one x row (j, k) of the right-hand side reads: each pointer is
// the start of a row of nx values (in global or shared memory); rows of a
// plane beyond a wall are NULL.  Names: U = u(j, k), Ujm = u(j-1, k), Uu =
// u(j, k+1), Ud = u(j, k-1), Vdjp = v(j+1, k-1), Wujm = w(j-1, k+1), H1u
// = H_u^{n-1}(j, k), and so on.
template <typename T> struct RowSet {
    const T *U, *Ujm, *Ujp, *Uu, *Ud;
    const T *V, *Vjm, *Vjp, *Vu, *Vd, *Vdjp;
    const T *W, *Wjm, *Wjp, *Wu, *Wujm, *Wd;
    const T *P, *Pjm, *Pd;
    const T *H1u, *H1v, *H1w;
};

// The lane's CPL values of each stencil row (names as in RowSet).
template <typename T, int CPL> struct RowVals {
    T U[CPL], Ujm[CPL], Ujp[CPL], Uu[CPL], Ud[CPL];
    T V[CPL], Vjm[CPL], Vjp[CPL], Vu[CPL], Vd[CPL], Vdjp[CPL];
    T W[CPL], Wjm[CPL], Wjp[CPL], Wu[CPL], Wujm[CPL], Wd[CPL];
    T P[CPL], Pjm[CPL], Pd[CPL];
};

// the lane's values of every stencil row from rs (0 beyond a wall)
template <typename T, int CPL>
FSEI_D void rhs_row_load(const RowSet<T> &rs, const RhsCoef<T> &cf, int i0, RowVals<T, CPL> &x) {
    const T z0 = T(0);
    ldrow(x.U, rs.U + i0); ldrow(x.Ujm, rs.Ujm + i0); ldrow(x.Ujp, rs.Ujp + i0);
    ldrow(x.V, rs.V + i0); ldrow(x.Vjm, rs.Vjm + i0); ldrow(x.Vjp, rs.Vjp + i0);
    ldrow(x.W, rs.W + i0); ldrow(x.Wjm, rs.Wjm + i0); ldrow(x.Wjp, rs.Wjp + i0);
    ldrow(x.P, rs.P + i0); ldrow(x.Pjm, rs.Pjm + i0);
    if (cf.hasup) {
        ldrow(x.Uu, rs.Uu + i0); ldrow(x.Vu, rs.Vu + i0);
        ldrow(x.Wu, rs.Wu + i0); ldrow(x.Wujm, rs.Wujm + i0);
    } else {
#pragma unroll
        for (int e = 0; e < CPL; ++e) x.Uu[e] = x.Vu[e] = x.Wu[e] = x.Wujm[e] = z0;
    }
    if (cf.hasdn) {
        ldrow(x.Ud, rs.Ud + i0); ldrow(x.Vd, rs.Vd + i0); ldrow(x.Vdjp, rs.Vdjp + i0);
        ldrow(x.Wd, rs.Wd + i0); ldrow(x.Pd, rs.Pd + i0);
    } else {
#pragma unroll
        for (int e = 0; e < CPL; ++e) x.Ud[e] = x.Vd[e] = x.Vdjp[e] = x.Wd[e] = x.Pd[e] = z0;
    }
}

// rhs_row_body on stencil values already in registers (x); rs gives the
// rows in memory for the x neighbours across a warp boundary and the
// H^{n-1} rows
template <typename T, int CPL, int LPR>
FSEI_D void rhs_row_compute(const GridDev &g, const Fields<T> &F, const RowSet<T> &rs,
                            const RowVals<T, CPL> &x, T *__restrict__ q0, T *__restrict__ q1,
                            T *__restrict__ q2, const StepScalars *sc, const RhsCoef<T> &cf,
                            int oc, int i0, T *xs) {
    const int nx = g.nx;
    const bool hasdn = cf.hasdn, hasup = cf.hasup;
    const T z0 = T(0), two = T(2);
    const T qidx = T(0.25) * cf.idx, qidy = T(0.25) * cf.idy, qidz = T(0.25) * cf.idzk,
            qihc = T(0.25) * cf.ihck;
    const T(&U)[CPL] = x.U, (&Ujm)[CPL] = x.Ujm, (&Ujp)[CPL] = x.Ujp, (&Uu)[CPL] = x.Uu,
          (&Ud)[CPL] = x.Ud;
    const T(&V)[CPL] = x.V, (&Vjm)[CPL] = x.Vjm, (&Vjp)[CPL] = x.Vjp, (&Vu)[CPL] = x.Vu,
          (&Vd)[CPL] = x.Vd, (&Vdjp)[CPL] = x.Vdjp;
    const T(&W)[CPL] = x.W, (&Wjm)[CPL] = x.Wjm, (&Wjp)[CPL] = x.Wjp, (&Wu)[CPL] = x.Wu,
          (&Wujm)[CPL] = x.Wujm, (&Wd)[CPL] = x.Wd;
    const T(&P)[CPL] = x.P, (&Pjm)[CPL] = x.Pjm, (&Pd)[CPL] = x.Pd;
    // x neighbours outside the lane's cells
    const T Ul = xnb<T, LPR, 1>(U[CPL - 1], rs.U, i0, nx, CPL);
    const T Ur = xnb<T, LPR, 0>(U[0], rs.U, i0, nx, CPL);
    const T Ujmr = xnb<T, LPR, 0>(Ujm[0], rs.Ujm, i0, nx, CPL);
    const T Udr = hasdn ? xnb<T, LPR, 0>(Ud[0], rs.Ud, i0, nx, CPL) : z0;
    const T Vl = xnb<T, LPR, 1>(V[CPL - 1], rs.V, i0, nx, CPL);
    const T Vr = xnb<T, LPR, 0>(V[0], rs.V, i0, nx, CPL);
    const T Vjpl = xnb<T, LPR, 1>(Vjp[CPL - 1], rs.Vjp, i0, nx, CPL);
    const T Wl = xnb<T, LPR, 1>(W[CPL - 1], rs.W, i0, nx, CPL);
    const T Wr = xnb<T, LPR, 0>(W[0], rs.W, i0, nx, CPL);
    const T Wul = hasup ? xnb<T, LPR, 1>(Wu[CPL - 1], rs.Wu, i0, nx, CPL) : z0;
    const T Pl = xnb<T, LPR, 1>(P[CPL - 1], rs.P, i0, nx, CPL);
    // at the CPL + 1 x faces / edges i0 .. i0+CPL of the lane: (u_{i-1} +
    // u_i)^2 and the products behind the xy and xz edge fluxes
    T usq[CPL + 1], pxy[CPL + 1], pxz[CPL + 1];
#pragma unroll
    for (int e = 0; e <= CPL; ++e) {
        const T um = e == 0 ? Ul : U[e - 1], u0 = e == CPL ? Ur : U[e];
        const T vm = e == 0 ? Vl : V[e - 1], v0 = e == CPL ? Vr : V[e];
        const T wm = e == 0 ? Wl : W[e - 1], w0 = e == CPL ? Wr : W[e];
        const T ujm = e == CPL ? Ujmr : Ujm[e], ud = e == CPL ? Udr : Ud[e];
        const T us = um + u0;
        usq[e] = us * us;
        pxy[e] = (v0 + vm) * (u0 + ujm);
        pxz[e] = hasdn ? (w0 + wm) * (u0 + ud) : z0;
    }
    T R[3][CPL];
    T Hn[3][CPL];
    const T *fx = F.fx ? F.fx + oc : nullptr, *fy = F.fy ? F.fy + oc : nullptr;
    const T *fz = (F.fz && !cf.wall_face) ? F.fz + oc : nullptr;
    {
        T H1[CPL], f[CPL];
        ldrow(H1, rs.H1u + i0);
        if (fx) ldrow(f, fx + i0);
#pragma unroll
        for (int e = 0; e < CPL; ++e) {
            const T uim = e == 0 ? Ul : U[e - 1], uip = e == CPL - 1 ? Ur : U[e + 1];
            const T vjpim = e == 0 ? Vjpl : Vjp[e - 1];
            const T wuim = e == 0 ? Wul : Wu[e - 1];
            const T pxy_jp = (Vjp[e] + vjpim) * (Ujp[e] + U[e]);
            const T pxz_kp = hasup ? (Wu[e] + wuim) * (Uu[e] + U[e]) : z0;
            const T Hu = -((usq[e + 1] - usq[e]) * qidx + (pxy_jp - pxy[e]) * qidy +
                           (pxz_kp - pxz[e]) * qidz);
            const T Lu = (uip - two * U[e] + uim) * cf.idx2 +
                         (Ujp[e] - two * U[e] + Ujm[e]) * cf.idy2 +
                         ((Uu[e] - U[e]) * cf.ihcu - (U[e] - Ud[e]) * cf.ihck) * cf.idzk;
            const T pim = e == 0 ? Pl : P[e - 1];
            Hn[0][e] = Hu;
            R[0][e] = cf.dt * (cf.gam * Hu + cf.rho * H1[e] + cf.inv_re * Lu -
                               (P[e] - pim) * cf.idx + (fx ? f[e] : z0) + cf.fc0);
        }
    }
    {
        T H1[CPL], f[CPL];
        ldrow(H1, rs.H1v + i0);
        if (fy) ldrow(f, fy + i0);
#pragma unroll
        for (int e = 0; e < CPL; ++e) {
            const T vim = e == 0 ? Vl : V[e - 1], vip = e == CPL - 1 ? Vr : V[e + 1];
            const T pyz = hasdn ? (W[e] + Wjm[e]) * (V[e] + Vd[e]) : z0;
            const T pyz_kp = hasup ? (Wu[e] + Wujm[e]) * (Vu[e] + V[e]) : z0;
            const T sp = V[e] + Vjp[e], sm = Vjm[e] + V[e];
            const T Hv = -((pxy[e + 1] - pxy[e]) * qidx + (sp * sp - sm * sm) * qidy +
                           (pyz_kp - pyz) * qidz);
            const T Lv = (vip - two * V[e] + vim) * cf.idx2 +
                         (Vjp[e] - two * V[e] + Vjm[e]) * cf.idy2 +
                         ((Vu[e] - V[e]) * cf.ihcu - (V[e] - Vd[e]) * cf.ihck) * cf.idzk;
            Hn[1][e] = Hv;
            R[1][e] = cf.dt * (cf.gam * Hv + cf.rho * H1[e] + cf.inv_re * Lv -
                               (P[e] - Pjm[e]) * cf.idy + (fy ? f[e] : z0) + cf.fc1);
        }
    }
    {
        T H1[CPL], f[CPL];
        ldrow(H1, rs.H1w + i0);
        if (fz) ldrow(f, fz + i0);
#pragma unroll
        for (int e = 0; e < CPL; ++e) {
            T Hw = z0, rw = z0;
            if (!cf.wall_face) {
                const T wim = e == 0 ? Wl : W[e - 1], wip = e == CPL - 1 ? Wr : W[e + 1];
                const T pyz = hasdn ? (W[e] + Wjm[e]) * (V[e] + Vd[e]) : z0;
                const T pyz_jp = hasdn ? (Wjp[e] + W[e]) * (Vjp[e] + Vdjp[e]) : z0;
                const T sp = W[e] + Wu[e], sm = Wd[e] + W[e];
                Hw = -((pxz[e + 1] - pxz[e]) * qidx + (pyz_jp - pyz) * qidy +
                       (sp * sp - sm * sm) * qihc);
                const T Lw = (wip - two * W[e] + wim) * cf.idx2 +
                             (Wjp[e] - two * W[e] + Wjm[e]) * cf.idy2 +
                             ((Wu[e] - W[e]) * cf.idzk - (W[e] - Wd[e]) * cf.idzd) * cf.ihck;
                rw = cf.dt * (cf.gam * Hw + cf.rho * H1[e] + cf.inv_re * Lw -
                              (P[e] - Pd[e]) * cf.ihck + (fz ? f[e] : z0) + cf.fc2);
            }
            Hn[2][e] = Hw;
            R[2][e] = rw;
        }
    }
    // the explicit extra term (the non-Newtonian remainder), if any, joins
    // H and, weighted dt gamma, the right-hand side
    if (F.hx) {
        const T dg = cf.dt * cf.gam;
        const T *ex[3] = {F.hx, F.hy, cf.wall_face ? nullptr : F.hz};
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            if (!ex[m]) continue;
            T X[CPL];
            ldrow(X, ex[m] + oc + i0);
#pragma unroll
            for (int e = 0; e < CPL; ++e) {
                Hn[m][e] += X[e];
                R[m][e] += dg * X[e];
            }
        }
    }
    // every load above precedes the first store (the row pointers may alias
    // the outputs as far as the compiler knows)
    strow(F.hu + oc + i0, Hn[0]);
    strow(F.hv + oc + i0, Hn[1]);
    strow(F.hw + oc + i0, Hn[2]);
    line_solve_uni<T, CPL, LPR, 3>(R, fpick<T>(sc->ax, sc->fax), fpick<T>(sc->cix, sc->fcix),
                                   sizeof(T) == 4 ? sc->ndecx_f : sc->ndecx_d, xs);
    strow(q0 + oc + i0, R[0]);
    strow(q1 + oc + i0, R[1]);
    strow(q2 + oc + i0, R[2]);
}

// H^n and the right-hand side of one x row at the lane's CPL cells (i0 ..),
// H^n stored to F.hu/hv/hw, then (I - beta L_x) q = RHS solved on the
// registers (line_solve_uni) and q stored to q0, q1, q2 (oc: offset of the
// row in the fields).  The products of two two-point averages are formed
// without their factors 1/2; the 1/4 is folded into the difference
// coefficients (scaling by powers of two is exact, so the values are those
// of rhs_point).  Edge products shared by two cells of a lane are formed
// once.  Every thread of the block calls it (line solves wider than a warp
// synchronise the block).
template <typename T, int CPL, int LPR>
FSEI_D void rhs_row_body(const GridDev &g, const Fields<T> &F, const RowSet<T> &rs,
                         T *__restrict__ q0, T *__restrict__ q1, T *__restrict__ q2,
                         const StepScalars *sc, const RhsCoef<T> &cf, int oc, int i0, T *xs) {
    RowVals<T, CPL> x;
    rhs_row_load<T, CPL>(rs, cf, i0, x);
    rhs_row_compute<T, CPL, LPR>(g, F, rs, x, q0, q1, q2, sc, cf, oc, i0, xs);
}

}  // namespace
}  // namespace fsei
