// Batched tridiagonal solves in shared memory for the approximately
// factorised viscous step (Sec. 3.1: one tridiagonal system per direction,
// cyclic in the two periodic directions) and for the z systems of the
// pressure Poisson equation.
//
// Partitioned elimination.  Each line of n unknowns is cut into P chunks
// [s, e].  In a chunk the interior rows s+1..e-1 are eliminated downwards,
// which writes every interior unknown as
//     x_i = d~_i - a~_i x_s - c~_i x_{i+1},
// and an upward pass then gives x_{s+1} and x_{e-1} through the two chunk
// ends x_s, x_e alone.  Substituting those into the original rows s and e
// leaves a tridiagonal system in the 2P chunk ends (cyclic when the line is
// periodic: the periodic coupling of the original line becomes the corner
// coupling of the reduced one).  It is solved by one thread per line with
// Thomas' algorithm, plus a Sherman-Morrison correction when cyclic.  A last
// upward pass per chunk recovers the interior.  This is Gaussian
// elimination in another order; for the diagonally dominant matrices here
// it needs no pivoting, like the Thomas algorithm it replaces.
#pragma once
#include "common.cuh"

namespace fsei {

// 1/x: the hardware reciprocal approximation (a few ulp) in single
// precision, where it sits on the serial critical path of the eliminations;
// a plain division in double
FSEI_D float rcp(float x) { return __fdividef(1.0f, x); }
FSEI_D double rcp(double x) { return 1.0 / x; }

// y - a x for real or complex x, y and real a
template <typename T> FSEI_D T nmad(T a, T x, T y) { return y - a * x; }
template <typename T> FSEI_D cplx<T> nmad(T a, cplx<T> x, cplx<T> y) {
    return {y.re - a * x.re, y.im - a * x.im};
}
template <typename T> FSEI_D T scl(T a, T x) { return a * x; }
template <typename T> FSEI_D cplx<T> scl(T a, cplx<T> x) { return {a * x.re, a * x.im}; }
template <typename T> FSEI_D T addv(T a, T b) { return a + b; }
template <typename T> FSEI_D cplx<T> addv(cplx<T> a, cplx<T> b) { return a + b; }

// Shared-memory words needed by stage_plan for a plan of n unknowns and P
// chunks (factors, reduced LU, PCR multipliers of up to kPcrLevels levels).
FSEI_HD int plan_stage_words(int n, int P) {
    return 5 * n + 8 * P + 2 + 2 * kPcrLevels * 2 * P + 2 * P;
}

// Reduced system of one line solved by one warp with parallel cyclic
// reduction: m = 2P unknowns, a power of two <= 128; lane l holds unknowns
// l + 32 q (q < NQ = m / 32), or unknown l alone when m <= 32.  Level s =
// 2^lev adds pk1 times unknown i - s and pk2 times unknown i + s (indices
// mod m) to unknown i; a shift s = 32 q' + s' reads lane l -/+ s' of the
// same or the neighbouring register slot.  Every lane of the warp must call
// it.
template <typename T, int NQ>
__device__ __forceinline__ void pcr_warp_slots(T *r, const TriPlan<T> &pl, int lane) {
    constexpr int m = 32 * NQ;
    T x[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) x[q] = r[lane + 32 * q];
    // v[(q + d) mod NQ] without indexing registers at run time
    auto pick = [](const T (&v)[NQ], int q) {
        q &= NQ - 1;
        T o = v[0];
#pragma unroll
        for (int u = 1; u < NQ; ++u) o = q == u ? v[u] : o;
        return o;
    };
    for (int lev = 0; lev < pl.levels; ++lev) {
        const int s = 1 << lev, sq = s >> 5, sl = s & 31;
        T tm[NQ], tp[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            tm[q] = __shfl_sync(0xffffffffu, x[q], (lane - sl) & 31);
            tp[q] = __shfl_sync(0xffffffffu, x[q], (lane + sl) & 31);
        }
        // unknown i = lane + 32 q: i - s sits in slot q - sq of lane lane -
        // sl, one slot lower where that lane wraps below 0; i + s likewise
        const int dm = lane >= sl ? -sq : -sq - 1, dp = lane + sl < 32 ? sq : sq + 1;
        T nx[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int i = lane + 32 * q;
            nx[q] = x[q] + pl.pk1[lev * m + i] * pick(tm, q + dm) +
                    pl.pk2[lev * m + i] * pick(tp, q + dp);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) x[q] = nx[q];
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) r[lane + 32 * q] = x[q] * pl.pdinv[lane + 32 * q];
}

template <typename T>
__device__ __forceinline__ void pcr_warp_solve(T *r, const TriPlan<T> &pl, int lane) {
    const int m = 2 * pl.P;
    if (m == 64) {
        pcr_warp_slots<T, 2>(r, pl, lane);
        return;
    }
    if (m == 128) {
        pcr_warp_slots<T, 4>(r, pl, lane);
        return;
    }
    T x = lane < m ? r[lane] : T(0);
    for (int lev = 0; lev < pl.levels; ++lev) {
        const int s = 1 << lev;
        const T xm = __shfl_sync(0xffffffffu, x, (lane - s) & (m - 1));
        const T xp = __shfl_sync(0xffffffffu, x, (lane + s) & (m - 1));
        if (lane < m) x = x + pl.pk1[lev * m + lane] * xm + pl.pk2[lev * m + lane] * xp;
    }
    if (lane < m) r[lane] = x * pl.pdinv[lane];
}

// Solve the reduced systems of lines 0..nl-1 (line l at red + l * rs): one
// warp per line in turn when the plan has PCR multipliers, else one thread
// per line with Thomas' algorithm (plus Sherman-Morrison when cyclic).
template <typename T>
__device__ __forceinline__ void reduced_lines(T *red, int rs, int nl, const TriPlan<T> &pl) {
    if (pl.levels > 0) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const int nw = (blockDim.x + 31) >> 5;
        for (int l = wid; l < nl; l += nw) pcr_warp_solve(red + l * rs, pl, lane);
        return;
    }
    const int t = threadIdx.x;
    if (t < nl) {
        T *r = red + t * rs;
        const int m = 2 * pl.P;
        T y = pl.rinv[0] * r[0];
        r[0] = y;
        for (int j = 1; j < m; ++j) {
            y = pl.rinv[j] * (r[j] - pl.rlo[j] * y);
            r[j] = y;
        }
        for (int j = m - 2; j >= 0; --j) {
            y = r[j] - pl.rcp[j] * y;
            r[j] = y;
        }
        if (pl.cyclic) {
            const T f = pl.rsc[1] * (r[0] + pl.rsc[0] * r[m - 1]);
            for (int j = 0; j < m; ++j) r[j] -= pl.rz[j] * f;
        }
    }
}

// Copy a plan's factors into shared memory (every thread of the block calls
// it; ends with a barrier) and return a plan that points there.
template <typename T>
__device__ TriPlan<T> stage_plan(const TriPlan<T> &in, T *sm) {
    const int n = in.n, m = 2 * in.P;
    TriPlan<T> out = in;
    T *a = sm, *c = a + n, *inv = c + n, *at = inv + n, *ct = at + n;
    T *rlo = ct + n, *rinv = rlo + m, *rcp = rinv + m, *rz = rcp + m, *rsc = rz + m;
    T *pk1 = rsc + 2, *pk2 = pk1 + kPcrLevels * m, *pdinv = pk2 + kPcrLevels * m;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a[i] = in.a[i];
        c[i] = in.c[i];
        inv[i] = in.inv[i];
        at[i] = in.at[i];
        ct[i] = in.ct[i];
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        rlo[i] = in.rlo[i];
        rinv[i] = in.rinv[i];
        rcp[i] = in.rcp[i];
        rz[i] = in.cyclic ? in.rz[i] : T(0);
    }
    if (threadIdx.x < 2) rsc[threadIdx.x] = in.cyclic ? in.rsc[threadIdx.x] : T(0);
    if (in.levels > 0) {
        for (int i = threadIdx.x; i < in.levels * m; i += blockDim.x) {
            pk1[i] = in.pk1[i];
            pk2[i] = in.pk2[i];
        }
        for (int i = threadIdx.x; i < m; i += blockDim.x) pdinv[i] = in.pdinv[i];
    }
    __syncthreads();
    out.a = a; out.c = c; out.inv = inv; out.at = at; out.ct = ct;
    out.rlo = rlo; out.rinv = rinv; out.rcp = rcp; out.rz = rz; out.rsc = rsc;
    out.pk1 = pk1; out.pk2 = pk2; out.pdinv = pdinv;
    return out;
}

// Same elimination with a matrix that differs per line (the Poisson z
// systems, one per Fourier mode: real matrix, complex right-hand side).
// The factors are computed on the fly: fa, fc hold a~, c~ (layout of the
// data with strides fes, fls); rlo, rdi, rup, rr hold the reduced rows.
// Mat provides a(i), c(i) (real, line-independent) and b(l, i).
template <typename T, typename Mat>
__device__ void tri_fly_solve(cplx<T> *s, int es, int ls, T *fa, T *fc, int fes, int fls,
                              int nl, int n, int P, int cyclic, const Mat &M,
                              cplx<T> *rr, T *rlo, T *rdi, T *rup, int rs) {
    const int t = threadIdx.x;
    const bool active = t < nl * P;
    const int l = t % nl, p = t / nl;
    int s0 = 0, e0 = 0;
    cplx<T> *d = s + l * ls;
    T *A = fa + l * fls, *C = fc + l * fls;
    if (active) {
        s0 = chunk_start(p, n, P);
        e0 = chunk_start(p + 1, n, P) - 1;
        int i = s0 + 1;
        T inv = rcp(M.b(l, i));
        T at = M.a(i) * inv, ct = M.c(i) * inv;
        A[i * fes] = at;
        C[i * fes] = ct;
        cplx<T> prev = scl(inv, d[i * es]);
        d[i * es] = prev;
        for (i = s0 + 2; i < e0; ++i) {
            const T ai = M.a(i);
            inv = rcp(M.b(l, i) - ai * ct);
            at = -ai * at * inv;
            ct = M.c(i) * inv;
            A[i * fes] = at;
            C[i * fes] = ct;
            prev = scl(inv, nmad(ai, prev, d[i * es]));
            d[i * es] = prev;
        }
        cplx<T> dh = d[(e0 - 1) * es];
        T ah = A[(e0 - 1) * fes], ch = C[(e0 - 1) * fes];
        const cplx<T> dhe = dh;
        const T ahe = ah, che = ch;
        for (i = e0 - 2; i > s0; --i) {
            const T cti = C[i * fes];
            dh = nmad(cti, dh, d[i * es]);
            ah = A[i * fes] - cti * ah;
            ch = -cti * ch;
        }
        const T as = M.a(s0), cs = M.c(s0), ae = M.a(e0), ce = M.c(e0);
        const int jF = l * rs + 2 * p, jE = jF + 1;
        rlo[jF] = as;
        rdi[jF] = M.b(l, s0) - cs * ah;
        rup[jF] = -cs * ch;
        rr[jF] = nmad(cs, dh, d[s0 * es]);
        rlo[jE] = -ae * ahe;
        rdi[jE] = M.b(l, e0) - ae * che;
        rup[jE] = ce;
        rr[jE] = nmad(ae, dhe, d[e0 * es]);
    }
    __syncthreads();
    if (t < nl) {
        const int m = 2 * P, o = t * rs;
        T *lo = rlo + o, *di = rdi + o, *up = rup + o;
        cplx<T> *r = rr + o;
        T g = T(0), lo0 = lo[0];
        if (cyclic) {
            g = -di[0];
            di[0] -= g;
            di[m - 1] -= up[m - 1] * lo0 / g;
        }
        // forward: overwrite up[] with c', di[] with 1/den
        T inv = rcp(di[0]);
        di[0] = inv;
        up[0] *= inv;
        cplx<T> y = scl(inv, r[0]);
        r[0] = y;
        for (int j = 1; j < m; ++j) {
            inv = rcp(di[j] - lo[j] * up[j - 1]);
            di[j] = inv;
            up[j] *= inv;
            y = scl(inv, nmad(lo[j], y, r[j]));
            r[j] = y;
        }
        for (int j = m - 2; j >= 0; --j) {
            y = nmad(up[j], y, r[j]);
            r[j] = y;
        }
        if (cyclic) {
            // Sherman-Morrison: z = T^-1 u with u = (g, 0, ..., 0, c_{n-1}),
            // the last entry being the original corner coupling of the line.
            // z overwrites lo[] (each lo[j] is read before it is replaced).
            const T cl = M.c(n - 1);
            T z = g * di[0];
            lo[0] = z;
            for (int j = 1; j < m; ++j) {
                const T uj = (j == m - 1) ? cl : T(0);
                z = di[j] * (uj - lo[j] * z);
                lo[j] = z;
            }
            for (int j = m - 2; j >= 0; --j) {
                z = lo[j] - up[j] * z;
                lo[j] = z;
            }
            const T vl = lo0 / g;
            const T fac = rcp(T(1) + lo[0] + vl * lo[m - 1]);
            const cplx<T> f = scl(fac, addv(r[0], scl(vl, r[m - 1])));
            for (int j = 0; j < m; ++j) r[j] = nmad(lo[j], f, r[j]);
        }
    }
    __syncthreads();
    if (active) {
        const int jF = l * rs + 2 * p;
        const cplx<T> F = rr[jF], E = rr[jF + 1];
        d[s0 * es] = F;
        d[e0 * es] = E;
        cplx<T> x = E;
        for (int i = e0 - 1; i > s0; --i) {
            x = nmad(C[i * fes], x, nmad(A[i * fes], F, d[i * es]));
            d[i * es] = x;
        }
    }
    __syncthreads();
}

// ------------------------------------- constant-coefficient periodic lines --
// In the two uniform periodic directions every line has the same cyclic
// Toeplitz matrix  A = (1 + 2r) I - r (E + E^-1),  r = beta / h^2,
// E x_i = x_{i+1} (indices mod n).  It factors exactly as
//     A = c (I - alpha E)(I - alpha E^-1),
// c alpha = r, c (1 + alpha^2) = 1 + 2r, i.e.
//     c = ((1 + 2r) + sqrt(1 + 4r)) / 2,  alpha = r / c  (0 <= alpha < 1),
// so A^-1 y is two periodic first-order recurrences and a scaling:
//     z_i = y_i + alpha z_{i+1},   x'_i = z_i + alpha x'_{i-1},   x = x' / c.
// A line is cut into P chunks of consecutive unknowns (chunk p starts at
// chunk_start(p, n, P)).  Each recurrence runs inside every chunk from a zero
// carry; the true carries then follow from a cyclic recurrence over the
// chunks, e.g. for the first one Z_p = zf_p + alpha^len_p Z_{p+1} (Z_p the
// true value at the chunk's first unknown, zf_p the zero-carry one), and
// each element gets alpha^distance times its chunk's carry added.  This is
// the same inverse as the cyclic Thomas / Sherman-Morrison solve of the
// paper's scheme, evaluated in another order.

// Cyclic recurrences over the chunks of nl lines, one warp per group of
// 32 / P lines (chunk p of a line in lane p of a width-P segment, P a power
// of two <= 32).  v[l * P + p] holds the zero-carry end value of chunk p of
// line l and is replaced by the carry that chunk p needs:
//   BACK = 1:  Z_p = v_p + g_p Z_{p+1},  chunk p needs Z_{p+1}
//   BACK = 0:  X_p = v_p + g_p X_{p-1},  chunk p needs X_{p-1}
// with g_p = alpha^len_p and indices mod P.  Every thread of the block calls
// it (the shuffles need whole warps); a barrier must separate it from the
// writes of v and from the reads of the carries.
template <typename T, int BACK, int FIXED = 0>
__device__ __forceinline__ void uni_carries(T *v, int nl, int n, int P, T alpha) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (int)((blockDim.x + 31) >> 5);
    const int per = 32 / P;             // lines per warp
    const int p = lane & (P - 1), seg = lane / P;
    for (int l0 = wid * per; l0 < nl; l0 += nw * per) {
        const int l = l0 + seg;
        const bool on = l < nl;
        const int len = FIXED ? FIXED : chunk_start(p + 1, n, P) - chunk_start(p, n, P);
        T g = T(1), a = alpha;
        for (int e = len; e > 0; e >>= 1) {      // alpha^len by squaring
            if (e & 1) g *= a;
            a *= a;
        }
        T A = on ? v[l * P + p] : T(0), B = g;
        // scan of the affine maps Z -> A + B Z along the segment
        for (int s = 1; s < P; s <<= 1) {
            const T A2 = BACK ? __shfl_down_sync(0xffffffffu, A, s, P)
                              : __shfl_up_sync(0xffffffffu, A, s, P);
            const T B2 = BACK ? __shfl_down_sync(0xffffffffu, B, s, P)
                              : __shfl_up_sync(0xffffffffu, B, s, P);
            if (BACK ? (p + s < P) : (p >= s)) {
                A = A + B * A2;
                B = B * B2;
            }
        }
        // the composition over the whole cycle closes it: V = A / (1 - B)
        // at lane 0 (BACK) or lane P-1; then V_p = A_p + B_p V
        const int root = BACK ? 0 : P - 1;
        const T Ar = __shfl_sync(0xffffffffu, A, root, P);
        const T Br = __shfl_sync(0xffffffffu, B, root, P);
        const T V = Ar * rcp(T(1) - Br);
        const T mine = A + B * V;
        // carry of chunk p: value of the next (BACK) or previous chunk
        const T nb = BACK ? __shfl_down_sync(0xffffffffu, mine, 1, P)
                          : __shfl_up_sync(0xffffffffu, mine, 1, P);
        const T carry = BACK ? (p == P - 1 ? V : nb) : (p == 0 ? V : nb);
        if (on) v[l * P + p] = carry;
    }
}

// Solve the chunks of nl constant-coefficient periodic lines, chunk p of
// line l held by one thread in d[0 .. len-1] (active threads only).  car:
// shared scratch of 2 nl P values.  EXACT: every chunk has L unknowns (len
// is then L; no per-unknown guards).  Every thread of the block calls it;
// it contains barriers.
template <typename T, int L, bool EXACT = false>
__device__ __forceinline__ void uni_solve(T (&d)[L], int len_, bool active, int l, int p, int nl,
                                          int n, int P, T alpha, T cinv, T *car) {
    const int len = EXACT ? L : len_;
    T *zc = car, *xc = car + nl * P;
    if (active) {
        T z = T(0);
#pragma unroll
        for (int i = L - 1; i >= 0; --i)
            if (i < len) {
                z = d[i] + alpha * z;
                d[i] = z;
            }
        zc[l * P + p] = z;          // zero-carry value at the chunk's first unknown
    }
    __syncthreads();
    uni_carries<T, 1, EXACT ? L : 0>(zc, nl, n, P, alpha);
    __syncthreads();
    if (active) {
        T pw = zc[l * P + p];       // Z of the next chunk
#pragma unroll
        for (int i = L - 1; i >= 0; --i)
            if (i < len) {
                pw *= alpha;
                d[i] += pw;
            }
        T x = T(0);
#pragma unroll
        for (int i = 0; i < L; ++i)
            if (i < len) {
                x = d[i] + alpha * x;
                d[i] = x;
            }
        xc[l * P + p] = x;          // zero-carry value at the chunk's last unknown
    }
    __syncthreads();
    uni_carries<T, 0, EXACT ? L : 0>(xc, nl, n, P, alpha);
    __syncthreads();
    if (active) {
        T pw = xc[l * P + p];       // X of the previous chunk
#pragma unroll
        for (int i = 0; i < L; ++i)
            if (i < len) {
                pw *= alpha;
                d[i] = (d[i] + pw) * cinv;
            }
    }
}

// ------------------------------------------ lane-resident periodic lines --
// A periodic line of n = LPR CPL unknowns held in registers by LPR
// consecutive threads (lane r of the line holds unknowns CPL r .. CPL r +
// CPL - 1); LPR a power of two.  A line of more than 32 lanes spans LPR / 32
// whole warps of the block.

// Carries of NV independent cyclic first-order recurrences with a common
// slope over the lanes of a line.  Lane p holds the zero-carry end values
// v[m] of its unknowns and g = alpha^CPL:
//   BACK = 1:  Z_p = v_p + g Z_{p+1}   (Z_p: value at lane p's first
//              unknown); on return v[m] = Z_{p+1}, the carry lane p needs
//   BACK = 0:  X_p = v_p + g X_{p-1}   (X_p: value at its last unknown);
//              on return v[m] = X_{p-1}
// with lane indices mod LPR.  Within a warp a scan of the affine maps Z ->
// v + g Z gives each lane the composition of its segment's maps; lines
// longer than a warp combine the warps' compositions through xs (2 NV
// values per warp of the block) between two barriers.  Every thread of the
// block calls it.
template <typename T, int LPR, int BACK, int NV>
FSEI_D void line_carries(T (&v)[NV], T g, T *xs) {
    constexpr int W = LPR < 32 ? LPR : 32;
    const int lane = threadIdx.x & 31;
    const int p = lane & (W - 1);
    T A[NV], B = g;
#pragma unroll
    for (int m = 0; m < NV; ++m) A[m] = v[m];
#pragma unroll
    for (int s = 1; s < W; s <<= 1) {
        const T B2 = BACK ? __shfl_down_sync(0xffffffffu, B, s, W)
                          : __shfl_up_sync(0xffffffffu, B, s, W);
        const bool take = BACK ? (p + s < W) : (p >= s);
#pragma unroll
        for (int m = 0; m < NV; ++m) {
            const T A2 = BACK ? __shfl_down_sync(0xffffffffu, A[m], s, W)
                              : __shfl_up_sync(0xffffffffu, A[m], s, W);
            if (take) A[m] = A[m] + B * A2;
        }
        if (take) B = B * B2;
    }
    // (A, B) at lane p: composition of the maps p .. W-1 (BACK) or 0 .. p
    // of its segment; the segment's own composition sits at its root lane
    const int root = BACK ? 0 : W - 1;
    T Vin[NV];   // value entering the segment from beyond its far end
    if (LPR <= 32) {
        const T Br = __shfl_sync(0xffffffffu, B, root, W);
#pragma unroll
        for (int m = 0; m < NV; ++m) {
            const T Ar = __shfl_sync(0xffffffffu, A[m], root, W);
            Vin[m] = Ar * rcp(T(1) - Br);   // the cycle closes: V = Ar + Br V
        }
    } else {
        constexpr int NW = LPR / 32;
        const int wid = threadIdx.x >> 5;
        const int w = wid & (NW - 1), w0 = wid - w;
        if (lane == root) {
#pragma unroll
            for (int m = 0; m < NV; ++m) xs[(2 * NV) * wid + m] = A[m];
            xs[(2 * NV) * wid + NV] = B;
        }
        __syncthreads();
        // compositions of the line's warps: around the whole cycle (TA, TB)
        // and over the warps beyond this one (RA, RB), BACK: w+1 .. NW-1,
        // forward: w-1 .. 0, each applied first-to-last away from the root
        T TA[NV], RA[NV], TB = T(1), RB = T(1);
#pragma unroll
        for (int m = 0; m < NV; ++m) { TA[m] = T(0); RA[m] = T(0); }
#pragma unroll
        for (int t = 0; t < NW; ++t) {
            // BACK composes from the last warp down to the first; forward
            // from the first up to the last
            const int u = BACK ? NW - 1 - t : t;
            const T *a = xs + (2 * NV) * (w0 + u);
            const T ub = a[NV];
#pragma unroll
            for (int m = 0; m < NV; ++m) TA[m] = a[m] + ub * TA[m];
            TB = ub * TB;
            if (BACK ? (u > w) : (u < w)) {
#pragma unroll
                for (int m = 0; m < NV; ++m) RA[m] = a[m] + ub * RA[m];
                RB = ub * RB;
            }
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < NV; ++m) {
            const T V = TA[m] * rcp(T(1) - TB);   // Z_0 (BACK) or X_{n-1}
            Vin[m] = RA[m] + RB * V;
        }
    }
    // value at this lane's own end, then the carry from its neighbour
#pragma unroll
    for (int m = 0; m < NV; ++m) {
        const T mine = A[m] + B * Vin[m];
        const T nb = BACK ? __shfl_down_sync(0xffffffffu, mine, 1, W)
                          : __shfl_up_sync(0xffffffffu, mine, 1, W);
        v[m] = (BACK ? p == W - 1 : p == 0) ? Vin[m] : nb;
    }
}

// The carries of line_carries where the slope decays fast: with |g|^D
// below the precision's tolerance (D <= kNearMax), Z_{p+1} (BACK) is
// sum_{k<D} g^k v_{p+1+k} and X_{p-1} is sum_{k<D} g^k v_{p-1-k} (lane
// indices mod LPR), the rest of the cyclic series dropped: each dropped
// term is at most |g|^D max|v|, and |g| <= 2^-4 makes their sum at most
// (16/15) |g|^D max|v|.  Lines within a warp read their neighbours by
// shuffles; longer ones through xs (NV values per thread of the block,
// BACK and forward in separate halves, so one barrier per call).  Every
// thread of the block calls it.
constexpr int kNearMax = 8;
template <typename T, int LPR, int BACK, int NV>
FSEI_D void line_carries_near(T (&v)[NV], T g, int D, T *xs) {
    if (LPR <= 32) {
        constexpr int W = LPR;
        const int p = threadIdx.x & (W - 1);
        T acc[NV];
#pragma unroll
        for (int m = 0; m < NV; ++m) acc[m] = T(0);
#pragma unroll
        for (int k = kNearMax - 1; k >= 0; --k) {
            if (k >= D) continue;   // uniform over the block
            const int src = BACK ? ((p + 1 + k) & (W - 1)) : ((p - 1 - k) & (W - 1));
#pragma unroll
            for (int m = 0; m < NV; ++m)
                acc[m] = __shfl_sync(0xffffffffu, v[m], src, W) + g * acc[m];
        }
#pragma unroll
        for (int m = 0; m < NV; ++m) v[m] = acc[m];
    } else {
        const int nt = (int)blockDim.x;
        const int r = (int)threadIdx.x & (LPR - 1), base = (int)threadIdx.x - r;
        T *buf = xs + (BACK ? 0 : NV * nt);
#pragma unroll
        for (int m = 0; m < NV; ++m) buf[m * nt + threadIdx.x] = v[m];
        __syncthreads();
        T acc[NV];
#pragma unroll
        for (int m = 0; m < NV; ++m) acc[m] = T(0);
#pragma unroll
        for (int k = kNearMax - 1; k >= 0; --k) {
            if (k >= D) continue;
            const int src = base + (BACK ? ((r + 1 + k) & (LPR - 1)) : ((r - 1 - k) & (LPR - 1)));
#pragma unroll
            for (int m = 0; m < NV; ++m) acc[m] = buf[m * nt + src] + g * acc[m];
        }
#pragma unroll
        for (int m = 0; m < NV; ++m) v[m] = acc[m];
    }
}

// Solve NV constant-coefficient periodic lines (I - beta L) x = y with the
// factorised inverse of uni_solve: z_i = y_i + alpha z_{i+1}, x'_i = z_i +
// alpha x'_{i-1}, x = x' / c, each recurrence evaluated lane by lane from a
// zero carry and corrected with the carries of line_carries.  d[m][e]:
// unknown CPL r + e of line m at lane r of the line.  ndec: the decay
// length of alpha (the least n with |alpha|^n below the precision's
// tolerance); where ndec / CPL lanes are at most kNearMax the carries take
// line_carries_near (xs: 2 NV values per thread of the block), else the
// exact scan (xs: 2 NV values per warp).  Every thread of the block calls
// it.
template <typename T, int CPL, int LPR, int NV>
FSEI_D void line_solve_uni(T (&d)[NV][CPL], T alpha, T cinv, int ndec, T *xs) {
    T g = T(1), a = alpha;
#pragma unroll
    for (int e = CPL; e > 0; e >>= 1) {    // alpha^CPL by squaring
        if (e & 1) g *= a;
        a *= a;
    }
    int D = (ndec + CPL - 1) / CPL;
    if (D < 1) D = 1;
    const bool near = D <= kNearMax;   // uniform over the grid
    T c[NV];
#pragma unroll
    for (int m = 0; m < NV; ++m) {
        T z = T(0);
#pragma unroll
        for (int i = CPL - 1; i >= 0; --i) {
            z = d[m][i] + alpha * z;
            d[m][i] = z;
        }
        c[m] = z;
    }
    if (near) line_carries_near<T, LPR, 1, NV>(c, g, D, xs);
    else line_carries<T, LPR, 1, NV>(c, g, xs);
#pragma unroll
    for (int m = 0; m < NV; ++m) {
        T pw = c[m];
#pragma unroll
        for (int i = CPL - 1; i >= 0; --i) {
            pw *= alpha;
            d[m][i] += pw;
        }
        T x = T(0);
#pragma unroll
        for (int i = 0; i < CPL; ++i) {
            x = d[m][i] + alpha * x;
            d[m][i] = x;
        }
        c[m] = x;
    }
    if (near) line_carries_near<T, LPR, 0, NV>(c, g, D, xs);
    else line_carries<T, LPR, 0, NV>(c, g, xs);
#pragma unroll
    for (int m = 0; m < NV; ++m) {
        T pw = c[m];
#pragma unroll
        for (int i = 0; i < CPL; ++i) {
            pw *= alpha;
            d[m][i] = (d[m][i] + pw) * cinv;
        }
    }
}

}  // namespace fsei
