// Right-hand side + x sweep of one fractional step (Sec. 2.1, Eq. 3;
// Sec. 3.1, the x factor of the approximate factorisation) marched along y:
// the same arithmetic per grid row as the row-resident kernel (rhs_row.cuh),
// but each lane walks a strip of S consecutive rows j of one plane k.
//
//   k_rhs_x_march  a row j reads 20 stencil rows (u, v, w, p at j-1 .. j+1
//                  and at the planes k-1, k+1); 9 of them are rows of j-1's
//                  stencil too and carry over in registers, the other 11
//                  are copied by the lane itself (cp.async, its own 16 or
//                  32 bytes of each) into a two-stage shared buffer one row
//                  ahead, so their memory latency overlaps the previous
//                  row's arithmetic; the plane's coefficients are formed
//                  once per strip.
#include <string.h>

#include "kernels.cuh"
#include "rhs_row.cuh"
#include "tri.cuh"

namespace fsei {

namespace {

// stencil rows of row j that are not rows of row j-1's stencil: slots of
// the staging buffer
enum MarchSlot {
    MS_UJP, MS_VJP, MS_WJP,   // u, v, w (j+1, k)
    MS_P,                     // p (j, k)
    MS_UU, MS_VU, MS_WU,      // u, v, w (j, k+1)
    MS_UD, MS_VDJP, MS_WD,    // u (j, k-1), v (j+1, k-1), w (j, k-1)
    MS_PD,                    // p (j, k-1)
    MS_COUNT
};

// the lane's CPL values (16 or 32 bytes) of a row, global -> shared
template <typename T, int CPL> FSEI_D void cp_chunk(T *dst, const T *src) {
    static_assert(CPL * sizeof(T) == 16 || CPL * sizeof(T) == 32, "16 or 32 bytes per lane");
    cp_async16(dst, src);
    if constexpr (CPL * sizeof(T) == 32) cp_async16(dst + 16 / sizeof(T), src + 16 / sizeof(T));
}

template <typename T, int CPL> FSEI_D void take(T (&d)[CPL], const T (&s)[CPL]) {
#pragma unroll
    for (int e = 0; e < CPL; ++e) d[e] = s[e];
}

// Lane layout as in k_rhs_x_row (LPR lanes per row, CPL cells per lane);
// the block's rpb row groups each march a strip of S rows, the block's
// strips consecutive in j.  Dynamic shared memory: 2 stages x MS_COUNT slots
// x blockDim lanes x CPL values, each lane reading only what it copied.
// Needs ny a multiple of rpb S.
template <typename T, int CPL, int LPR>
FSEI_D void
k_rhs_x_march(GridDev g, Fields<T> F, T *__restrict__ q0, T *__restrict__ q1,
              T *__restrict__ q2, const StepScalars *sc, int rpb, int S, T fc0, T fc1, T fc2,
              T inv_re) {
    extern __shared__ __align__(16) unsigned char march_smem[];
    // carries of the line solve (lines longer than a warp)
    __shared__ T xs[LPR > 32 ? 2 * 3 * (LPR > 128 ? LPR : 128) : 1];
    pdl_wait();
    pdl_trigger();
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int nt = (int)blockDim.x;
    const int nbs = ny / (rpb * S);
    const int k = blockIdx.x / nbs;
    const int jbeg = (blockIdx.x % nbs) * rpb * S + ((int)threadIdx.x / LPR) * S;
    const int i0 = ((int)threadIdx.x & (LPR - 1)) * CPL;
    const RhsCoef<T> cf = rhs_coef<T>(g, sc, k, fc0, fc1, fc2, inv_re);
    const int kd = k == 0 ? nz - 1 : k - 1, ku = k == nz - 1 ? 0 : k + 1;
    auto row = [&](const T *f, int kk, int jj) { return f + ((size_t)kk * ny + jj) * nx; };
    T *const mine = reinterpret_cast<T *>(march_smem) + (size_t)threadIdx.x * CPL;
    const int slot = nt * CPL, stage = MS_COUNT * nt * CPL;
    // copies of row jj's staged rows into stage s
    auto issue = [&](int jj, int s) {
        const int jjp = jj == ny - 1 ? 0 : jj + 1;
        T *d = mine + s * stage;
        cp_chunk<T, CPL>(d + MS_UJP * slot, row(F.u, k, jjp) + i0);
        cp_chunk<T, CPL>(d + MS_VJP * slot, row(F.v, k, jjp) + i0);
        cp_chunk<T, CPL>(d + MS_WJP * slot, row(F.w, k, jjp) + i0);
        cp_chunk<T, CPL>(d + MS_P * slot, row(F.p, k, jj) + i0);
        if (cf.hasup) {
            cp_chunk<T, CPL>(d + MS_UU * slot, row(F.u, ku, jj) + i0);
            cp_chunk<T, CPL>(d + MS_VU * slot, row(F.v, ku, jj) + i0);
            cp_chunk<T, CPL>(d + MS_WU * slot, row(F.w, ku, jj) + i0);
        }
        if (cf.hasdn) {
            cp_chunk<T, CPL>(d + MS_UD * slot, row(F.u, kd, jj) + i0);
            cp_chunk<T, CPL>(d + MS_VDJP * slot, row(F.v, kd, jjp) + i0);
            cp_chunk<T, CPL>(d + MS_WD * slot, row(F.w, kd, jj) + i0);
            cp_chunk<T, CPL>(d + MS_PD * slot, row(F.p, kd, jj) + i0);
        }
    };
    RowVals<T, CPL> x;
    {
        // the rows the strip's first row shares with the row before it;
        // rows beyond a wall are 0 for the whole strip
        const T z0 = T(0);
        const int jm = jbeg == 0 ? ny - 1 : jbeg - 1;
        ldrow(x.U, row(F.u, k, jbeg) + i0);
        ldrow(x.Ujm, row(F.u, k, jm) + i0);
        ldrow(x.V, row(F.v, k, jbeg) + i0);
        ldrow(x.Vjm, row(F.v, k, jm) + i0);
        ldrow(x.W, row(F.w, k, jbeg) + i0);
        ldrow(x.Wjm, row(F.w, k, jm) + i0);
        ldrow(x.Pjm, row(F.p, k, jm) + i0);
        if (cf.hasup) {
            ldrow(x.Wujm, row(F.w, ku, jm) + i0);
        } else {
#pragma unroll
            for (int e = 0; e < CPL; ++e) x.Uu[e] = x.Vu[e] = x.Wu[e] = x.Wujm[e] = z0;
        }
        if (cf.hasdn) {
            ldrow(x.Vd, row(F.v, kd, jbeg) + i0);
        } else {
#pragma unroll
            for (int e = 0; e < CPL; ++e) x.Ud[e] = x.Vd[e] = x.Vdjp[e] = x.Wd[e] = x.Pd[e] = z0;
        }
    }
    issue(jbeg, 0);
    cp_async_commit();
    for (int t = 0; t < S; ++t) {
        const int j = jbeg + t;
        if (t + 1 < S) issue(j + 1, (t + 1) & 1);
        cp_async_commit();
        cp_async_wait_prior();   // row j's copies have landed
        const T *d = mine + (t & 1) * stage;
        ldrow(x.Ujp, d + MS_UJP * slot);
        ldrow(x.Vjp, d + MS_VJP * slot);
        ldrow(x.Wjp, d + MS_WJP * slot);
        ldrow(x.P, d + MS_P * slot);
        if (cf.hasup) {
            ldrow(x.Uu, d + MS_UU * slot);
            ldrow(x.Vu, d + MS_VU * slot);
            ldrow(x.Wu, d + MS_WU * slot);
        }
        if (cf.hasdn) {
            ldrow(x.Ud, d + MS_UD * slot);
            ldrow(x.Vdjp, d + MS_VDJP * slot);
            ldrow(x.Wd, d + MS_WD * slot);
            ldrow(x.Pd, d + MS_PD * slot);
        }
        const int jp = j == ny - 1 ? 0 : j + 1, jm = j == 0 ? ny - 1 : j - 1;
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
        rhs_row_compute<T, CPL, LPR>(g, F, rs, x, q0, q1, q2, sc, cf, (k * ny + j) * nx, i0, xs);
        // row j + 1 shares these with row j
        take(x.Ujm, x.U);
        take(x.U, x.Ujp);
        take(x.Vjm, x.V);
        take(x.V, x.Vjp);
        take(x.Wjm, x.W);
        take(x.W, x.Wjp);
        take(x.Pjm, x.P);
        take(x.Wujm, x.Wu);
        take(x.Vd, x.Vdjp);
    }
}

}  // namespace

template <typename T, int CPL, int LPR>
constexpr Kernel<k_rhs_x_march<T, CPL, LPR>, (LPR > 128 ? LPR : 128),
                 (sizeof(T) == 4 && CPL == 4 ? 4 : 0)>
    K_rhs_x_march{};

// ------------------------------------------------------------- launchers --
namespace {

template <typename T> size_t march_smem_bytes(int cpl, int nthreads) {
    return 2 * (size_t)MS_COUNT * nthreads * cpl * sizeof(T);
}

template <typename T, int CPL, int LPR>
void march_launch(const GridDev &g, const Fields<T> &F, Work<T> &W, const StepScalars *sc,
                  const StepArgs &a, int rpb, int S, cudaStream_t st) {
    const int nt = rpb * LPR;
    K_rhs_x_march<T, CPL, LPR>.launch(W.pdl != 0, dim3(g.nz * (g.ny / (rpb * S))), dim3(nt),
                                      march_smem_bytes<T>(CPL, nt), st, g, F, W.q0, W.q1, W.q2,
                                      sc, rpb, S, T(a.fconst[0]), T(a.fconst[1]),
                                      T(a.fconst[2]), T(1.0 / a.re));
}

template <typename T, int CPL>
bool march_dispatch(const GridDev &g, const Fields<T> &F, Work<T> &W, const StepScalars *sc,
                    const StepArgs &a, int lpr, int rpb, int S, cudaStream_t st) {
    switch (lpr) {
    case 16: march_launch<T, CPL, 16>(g, F, W, sc, a, rpb, S, st); return true;
    case 32: march_launch<T, CPL, 32>(g, F, W, sc, a, rpb, S, st); return true;
    case 64: march_launch<T, CPL, 64>(g, F, W, sc, a, rpb, S, st); return true;
    case 128: march_launch<T, CPL, 128>(g, F, W, sc, a, rpb, S, st); return true;
    default: return false;
    }
}

}  // namespace

// The row layout of rhs_row_geometry with cpl cells per lane (0: its
// default), 16 or 32 bytes per lane, 16 to 128 lanes per row, and strips of
// S >= 2 rows that tile ny by rpb S.
template <typename T> bool rhs_march_geometry(const GridDev &g, int prefer, int S, int &cpl,
                                              int &lpr, int &rpb) {
    if (S < 2 || !rhs_row_geometry<T>(g, cpl, lpr, rpb, prefer)) return false;
    const int bytes = cpl * (int)sizeof(T);
    return (bytes == 16 || bytes == 32) && lpr >= 16 && lpr <= 128 && g.ny % (rpb * S) == 0;
}

bool rhs_strip_admissible(const GridDev &g, int elem_size, int cpl, int S) {
    int c = 0, l = 0, r = 0;
    const bool ok = elem_size == 4 ? rhs_march_geometry<float>(g, cpl, S, c, l, r)
                                   : rhs_march_geometry<double>(g, cpl, S, c, l, r);
    return ok && (cpl == 0 || c == cpl);
}

template <typename T>
bool launch_rhs_x_march(const GridDev &g, const Fields<T> &F, Work<T> &W, const StepScalars *sc,
                        const StepArgs &a, cudaStream_t st) {
    int cpl = 0, lpr = 0, rpb = 0;
    if (!rhs_march_geometry<T>(g, W.rhs_cpl, W.rhs_strip, cpl, lpr, rpb)) return false;
    if (cpl == 4) return march_dispatch<T, 4>(g, F, W, sc, a, lpr, rpb, W.rhs_strip, st);
    if constexpr (sizeof(T) == 4)
        if (cpl == 8) return march_dispatch<T, 8>(g, F, W, sc, a, lpr, rpb, W.rhs_strip, st);
    return false;
}

template <typename T> void set_smem_limits_march(const GridDev &g, const Work<T> &W) {
    (void)g;
    (void)W;
    raise_smem_limit(K_rhs_x_march<T, 4, 16>.solo());
    raise_smem_limit(K_rhs_x_march<T, 4, 32>.solo());
    raise_smem_limit(K_rhs_x_march<T, 4, 64>.solo());
    raise_smem_limit(K_rhs_x_march<T, 4, 128>.solo());
    if constexpr (sizeof(T) == 4) {
        raise_smem_limit(K_rhs_x_march<T, 8, 16>.solo());
        raise_smem_limit(K_rhs_x_march<T, 8, 32>.solo());
        raise_smem_limit(K_rhs_x_march<T, 8, 64>.solo());
        raise_smem_limit(K_rhs_x_march<T, 8, 128>.solo());
    }
}

#define FSEI_INST(T)                                                                           \
    template bool launch_rhs_x_march<T>(const GridDev &, const Fields<T> &, Work<T> &,         \
                                        const StepScalars *, const StepArgs &, cudaStream_t); \
    template void set_smem_limits_march<T>(const GridDev &, const Work<T> &);
FSEI_INST(float)
FSEI_INST(double)
#undef FSEI_INST

}  // namespace fsei
