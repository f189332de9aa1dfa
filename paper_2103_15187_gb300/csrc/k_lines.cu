// Implicit viscous sweeps along y and z (Sec. 3.1: one tridiagonal system
// per direction; cyclic in y; Dirichlet walls or cyclic in z).
//
// z lines (stretched mesh: the coefficients vary along the line) use the
// partitioned elimination of tri.cuh held in registers.  A block owns tx
// consecutive x columns of one component and one y row.  Thread (lane, p)
// owns chunk p of line lane: it loads the chunk straight from global memory
// (a warp reads tx consecutive x values per row: coalesced), eliminates the
// chunk interior in registers, writes its two reduced-row right-hand sides
// to shared memory, and after the reduced systems are solved recovers the
// interior in registers and stores it.  Shared memory holds only the plan
// factors and the reduced systems.
//
// y lines (uniform and periodic: one cyclic Toeplitz matrix for every line)
// use the factorised solve uni_solve of tri.cuh with the same block shape:
// chunks in registers, only the chunk carries pass through shared memory.
#include <string.h>

#include "kernels.cuh"
#include "tri.cuh"

namespace fsei {

namespace {

// The chunk's last rows are picked out with "i >= len - 1" style tests, never
// "i == len - 1": the compiler folds an equality chain over an unrolled loop
// into an array access at a run-time index, which moves d[] to local memory.
// Chunks hold at least three unknowns.
template <typename T, int L, int CX>
__device__ __forceinline__ void chunk_forward(T (&d)[CX][L], int len, const TriPlan<T> &pl,
                                              int s0, T (&rF)[CX], T (&rE)[CX]) {
    // interior rows 1 .. len-2 of the chunk (positions s0+1 .. s0+len-2);
    // the CX columns of the lane share every factor
    {
        const T inv = pl.inv[s0 + 1];
#pragma unroll
        for (int c = 0; c < CX; ++c) d[c][1] = inv * d[c][1];
    }
#pragma unroll
    for (int i = 2; i < L - 1; ++i)
        if (i < len - 1) {
            const T inv = pl.inv[s0 + i], a = pl.a[s0 + i];
#pragma unroll
            for (int c = 0; c < CX; ++c) d[c][i] = inv * (d[c][i] - a * d[c][i - 1]);
        }
    // upward pass for the right-hand side part of x_{s0+1}; dh starts at 0,
    // so at i = len-2 it takes d[len-2]
    T dh[CX], dhe[CX], last[CX];
#pragma unroll
    for (int c = 0; c < CX; ++c) dh[c] = dhe[c] = last[c] = T(0);
#pragma unroll
    for (int i = L - 2; i >= 1; --i) {
        const T ct = pl.ct[s0 + i];
#pragma unroll
        for (int c = 0; c < CX; ++c) {
            if (i >= len - 2) dhe[c] = d[c][i];
            if (i <= len - 2) dh[c] = d[c][i] - ct * dh[c];
        }
    }
#pragma unroll
    for (int i = 0; i < L; ++i)
        if (i <= len - 1) {
#pragma unroll
            for (int c = 0; c < CX; ++c) last[c] = d[c][i];
        }
    const T c0 = pl.c[s0], ae = pl.a[s0 + len - 1];
#pragma unroll
    for (int c = 0; c < CX; ++c) {
        rF[c] = d[c][0] - c0 * dh[c];
        rE[c] = last[c] - ae * dhe[c];
    }
}

template <typename T, int L, int CX>
__device__ __forceinline__ void chunk_backward(T (&d)[CX][L], int len, const TriPlan<T> &pl,
                                               int s0, const T (&F)[CX], const T (&E)[CX]) {
    T x[CX];
#pragma unroll
    for (int c = 0; c < CX; ++c) {
        d[c][0] = F[c];
        x[c] = E[c];
    }
#pragma unroll
    for (int i = L - 1; i >= 1; --i) {
        if (i >= len - 1) {
#pragma unroll
            for (int c = 0; c < CX; ++c) d[c][i] = E[c];   // rows past the chunk are not stored
        } else {
            const T at = pl.at[s0 + i], ct = pl.ct[s0 + i];
#pragma unroll
            for (int c = 0; c < CX; ++c) {
                x[c] = d[c][i] - at * F[c] - ct * x[c];
                d[c][i] = x[c];
            }
        }
    }
}

// DIR 1: y lines of plane k.  DIR 2: z lines of row j.
// MODE (z only): 0 -> q = u^n + solution (step); 1 -> q = W solution
// (adjoint, W = dz_k for u, v and hc_k for w).
// Blocks hold at most 256 threads for chunks of <= 16 unknowns, 512 above
// (sweep_geometry); the minimum-blocks hint leaves room for the chunk, and in
// single precision for the prefetched u^n, in registers.
// EXACT: every chunk of the line holds L unknowns (n = L P).
// CX: x columns per lane (1, or 2 as one 8- or 16-byte vector per row): the
// chunk's factors, read from shared memory once per row, serve both, and a
// warp's loads cover 2 tx consecutive columns.
// whether a register sweep of chunks of L rows stages its plan in shared
// memory (sweep_reg_body)
template <int L> constexpr bool kStagePlan = L <= 16;

template <typename T, int CX> struct ColVec;
template <typename T> struct ColVec<T, 1> { T v[1]; };
template <typename T> struct alignas(2 * sizeof(T)) ColVec<T, 2> { T v[2]; };

template <typename T, int L, int DIR, int MODE, bool EXACT, int CX>
__device__ __forceinline__ void sweep_reg_body(const GridDev &g, const Fields<T> &F,
                                               T *__restrict__ q0, T *__restrict__ q1,
                                               T *__restrict__ q2, const TriPlan<T> &pa,
                                               const TriPlan<T> &pb, int tx, T *sm) {
    using V = ColVec<T, CX>;
    const int nx = g.nx, ny = g.ny;
    const int nxt = (nx + tx * CX - 1) / (tx * CX);
    int b = blockIdx.x;
    const int xt = b % nxt;
    b /= nxt;
    const int outer = DIR == 1 ? g.nz : g.ny;
    const int row = b % outer;          // k for y lines, j for z lines
    const int comp = b / outer;
    const TriPlan<T> &src = (DIR == 2 && comp == 2) ? pb : pa;
    const int Pmax = pa.P > pb.P ? pa.P : pb.P;
    const int rs = 2 * Pmax + 1;
    T *red = sm;
    T *q = comp == 0 ? q0 : (comp == 1 ? q1 : q2);
    const size_t stride = DIR == 1 ? (size_t)nx : (size_t)nx * ny;
    const int t = threadIdx.x;
    const int l = t % tx, p = t / tx;
    const int x = (xt * tx + l) * CX;   // nx is even, so x < nx covers the pair
    const bool active = p < src.P && x < nx;
    const size_t base = (DIR == 1 ? (size_t)row * ny * nx : (size_t)row * nx) + x +
                        (size_t)src.off * stride;
    int s0 = 0, len = 0;
    T d[CX][L];
    // u^n of the step's z sweep is prefetched with the chunk in single
    // precision (in double it would cost the registers of a second chunk)
    constexpr bool kPrefetch = DIR == 2 && MODE == 0 && sizeof(T) == 4;
    V un_pre[kPrefetch ? L : 1];
    // issue the chunk's loads first; staging the plan below overlaps them
    // lastpad: the chunk ends with the plan's padding unknown (0, not stored)
    bool lastpad = false;
    auto keep = [&](int i) {
        return (EXACT || i < len) && !(lastpad && i == (EXACT ? L : len) - 1);
    };
    if (active) {
        s0 = EXACT ? p * L : chunk_start(p, src.n, src.P);
        len = EXACT ? L : chunk_start(p + 1, src.n, src.P) - s0;
        lastpad = src.pad && s0 + (EXACT ? L : len) == src.n;
        const T *qp = q + base + (size_t)s0 * stride;
#pragma unroll
        for (int i = 0; i < L; ++i) {
            V v;
            if (keep(i)) v = *reinterpret_cast<const V *>(qp + (size_t)i * stride);
            else for (int c = 0; c < CX; ++c) v.v[c] = T(0);
#pragma unroll
            for (int c = 0; c < CX; ++c) d[c][i] = v.v[c];
        }
        if constexpr (kPrefetch) {
            const T *un = comp == 0 ? F.u : (comp == 1 ? F.v : F.w);
            const T *up = un + base + (size_t)s0 * stride;
#pragma unroll
            for (int i = 0; i < L; ++i)
                if (keep(i)) un_pre[i] = *reinterpret_cast<const V *>(up + (size_t)i * stride);
        }
    }
    // chunks of up to 16 rows: the plan's factors staged in shared memory
    // once per block; longer chunks (the 768-row lines) read them through
    // the L1 cache instead -- their blocks are half as many again per line
    // and the staging of 768 rows' factors cost more than it saved (512 x
    // 512 x 768: 2.31 -> 2.16 ms; at 256^3 staging stays faster, 121
    // against 129 us)
    const TriPlan<T> pl = kStagePlan<L> ? stage_plan(src, red + (size_t)tx * CX * rs) : src;
    if (active) {
        T rF[CX], rE[CX];
        chunk_forward<T, L, CX>(d, EXACT ? L : len, pl, s0, rF, rE);
#pragma unroll
        for (int c = 0; c < CX; ++c) {
            red[(l * CX + c) * rs + 2 * p] = rF[c];
            red[(l * CX + c) * rs + 2 * p + 1] = rE[c];
        }
    }
    __syncthreads();
    reduced_lines<T>(red, rs, tx * CX, pl);
    __syncthreads();
    if (active) {
        T Fv[CX], Ev[CX];
#pragma unroll
        for (int c = 0; c < CX; ++c) {
            Fv[c] = red[(l * CX + c) * rs + 2 * p];
            Ev[c] = red[(l * CX + c) * rs + 2 * p + 1];
        }
        chunk_backward<T, L, CX>(d, EXACT ? L : len, pl, s0, Fv, Ev);
        T *qp = fresh(q) + base + (size_t)s0 * stride;
#pragma unroll
        for (int i = 0; i < L; ++i) {
            if (!keep(i)) continue;
            V v;
            if (DIR == 1) {
#pragma unroll
                for (int c = 0; c < CX; ++c) v.v[c] = d[c][i];
            } else if (MODE == 0) {
                V un;
                if constexpr (kPrefetch) {
                    un = un_pre[i];
                } else {
                    const T *unf = comp == 0 ? F.u : (comp == 1 ? F.v : F.w);
                    un = *reinterpret_cast<const V *>(unf + base + (size_t)(s0 + i) * stride);
                }
#pragma unroll
                for (int c = 0; c < CX; ++c) v.v[c] = un.v[c] + d[c][i];
            } else {
                const int k = s0 + i + pl.off;
                const T wk = comp < 2 ? Metric<T>::dz(g)[k] : T(1) / Metric<T>::ihc(g)[k];
#pragma unroll
                for (int c = 0; c < CX; ++c) v.v[c] = wk * d[c][i];
            }
            *reinterpret_cast<V *>(qp + (size_t)i * stride) = v;
        }
    }
}

template <typename T, int L, int DIR, int MODE, int CX>
FSEI_D void
k_sweep_reg(GridDev g, Fields<T> F, T *__restrict__ q0, T *__restrict__ q1,
            T *__restrict__ q2, TriPlan<T> pa, TriPlan<T> pb, int tx) {
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_wait();
    pdl_trigger();
    T *sm = reinterpret_cast<T *>(smraw);
    // the component of this block picks its plan; lines of L P unknowns take
    // the guard-free path
    const int outer = DIR == 1 ? g.nz : g.ny;
    const int comp = (int)blockIdx.x / ((g.nx + tx * CX - 1) / (tx * CX)) / outer;
    const TriPlan<T> &src = (DIR == 2 && comp == 2) ? pb : pa;
    if (src.n == L * src.P)
        sweep_reg_body<T, L, DIR, MODE, true, CX>(g, F, q0, q1, q2, pa, pb, tx, sm);
    else
        sweep_reg_body<T, L, DIR, MODE, false, CX>(g, F, q0, q1, q2, pa, pb, tx, sm);
}

// y sweep of plane k: q = (I - beta L_y)^-1 q for the three components.
// EXACT: every chunk holds L unknowns (ny = L P), no per-unknown guards.
// Single precision, L <= 16: 5 blocks per SM (48 registers, no spills;
// 256^3: 84 -> 79 us against 4 blocks).
template <typename T, int L, bool EXACT>
FSEI_D void
k_sweep_y_uni(GridDev g, T *__restrict__ q0, T *__restrict__ q1, T *__restrict__ q2,
              const StepScalars *sc, int P, int tx) {
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_wait();
    pdl_trigger();
    T *car = reinterpret_cast<T *>(smraw);
    const int nx = g.nx, ny = g.ny;
    const int nxt = (nx + tx - 1) / tx;
    int b = blockIdx.x;
    const int xt = b % nxt;
    b /= nxt;
    const int k = b % g.nz, comp = b / g.nz;
    T *q = comp == 0 ? q0 : (comp == 1 ? q1 : q2);
    const int t = threadIdx.x;
    const int p = ddiv(t, tx), l = t - p * tx;
    const int x = xt * tx + l;
    const bool active = p < P && x < nx;
    const int s0 = active ? (EXACT ? p * L : chunk_start(p, ny, P)) : 0;
    const int len = EXACT ? L : (active ? chunk_start(p + 1, ny, P) - s0 : 0);
    T *qp = q + (k * ny + s0) * nx + x;    // a field holds < 2^31 values
    T d[L];
#pragma unroll
    for (int i = 0; i < L; ++i)
        if (active && i < len) d[i] = qp[i * nx];
    uni_solve<T, L, EXACT>(d, len, active, l, p, tx, ny, P, fpick<T>(sc->ay, sc->fay),
                           fpick<T>(sc->ciy, sc->fciy), car);
    T *qs = fresh(qp);
#pragma unroll
    for (int i = 0; i < L; ++i)
        if (active && i < len) qs[i * nx] = d[i];
}

// the kernels with their launch bounds
// blocks per SM the z sweep is compiled for: room for the chunk (and in
// single precision the prefetched u^n) of CX columns in registers
constexpr int sweep_min_blocks(int L, int tsz, int CX) {
    return L > 16 ? 1 : (CX == 1 ? (tsz == 4 ? 3 : 2) : (tsz == 4 ? 2 : 1));
}
template <typename T, int L, int DIR, int MODE, int CX = 1>
constexpr Kernel<k_sweep_reg<T, L, DIR, MODE, CX>, (L <= 16 ? 256 : 512),
                 sweep_min_blocks(L, (int)sizeof(T), CX)>
    K_sweep_reg{};
template <typename T, int L, bool EXACT>
constexpr Kernel<k_sweep_y_uni<T, L, EXACT>, 256,
                 (L <= 16 ? (sizeof(T) == 4 ? 5 : 2) : (sizeof(T) == 4 ? 2 : 1))>
    K_sweep_y_uni{};

template <typename T, int L, int DIR, int MODE, int CX>
void launch_reg(const GridDev &g, const Fields<T> &F, Work<T> &W, const TriPlan<T> &pa,
                const TriPlan<T> &pb, int tx, cudaStream_t st) {
    const int Pmax = pa.P > pb.P ? pa.P : pb.P;
    const int nmax = pa.n > pb.n ? pa.n : pb.n;
    const int threads = ((tx * Pmax + 31) / 32) * 32;
    const size_t smem =
        sizeof(T) * ((size_t)tx * CX * (2 * Pmax + 1) +
                     (kStagePlan<L> ? plan_stage_words(nmax, Pmax) : 0));
    const int nxt = (g.nx + tx * CX - 1) / (tx * CX);
    const int outer = DIR == 1 ? g.nz : g.ny;
    K_sweep_reg<T, L, DIR, MODE, CX>.launch(W.pdl != 0, dim3(3 * outer * nxt), dim3(threads),
                                            smem, st, g, F, W.q0, W.q1, W.q2, pa, pb, tx);
}

template <typename T, int DIR, int MODE>
void dispatch(const GridDev &g, const Fields<T> &F, Work<T> &W, cudaStream_t st) {
    static_assert(DIR == 2, "y lines use k_sweep_y_uni");
    const TriPlan<T> &pa = W.plan[2];
    const TriPlan<T> &pb = W.plan[3];
    const int chunk = W.chunk_z;
    const int tx = W.tx_z;
    // two columns per lane (a schedule choice) for chunks of up to 16 rows
    if (W.zsw_cols == 2 && chunk <= 16) {
        if (chunk <= 8) launch_reg<T, 8, DIR, MODE, 2>(g, F, W, pa, pb, tx, st);
        else if (chunk == 12) launch_reg<T, 12, DIR, MODE, 2>(g, F, W, pa, pb, tx, st);
        else launch_reg<T, 16, DIR, MODE, 2>(g, F, W, pa, pb, tx, st);
        return;
    }
    // chunks of exactly 12 or 24 rows (nz = 192, 384, 768 ...) get registers
    // of their own length, so that those lines also take the guard-free path
    if (chunk <= 8) launch_reg<T, 8, DIR, MODE, 1>(g, F, W, pa, pb, tx, st);
    else if (chunk == 12) launch_reg<T, 12, DIR, MODE, 1>(g, F, W, pa, pb, tx, st);
    else if (chunk <= 16) launch_reg<T, 16, DIR, MODE, 1>(g, F, W, pa, pb, tx, st);
    else if (chunk == 24) launch_reg<T, 24, DIR, MODE, 1>(g, F, W, pa, pb, tx, st);
    else launch_reg<T, 32, DIR, MODE, 1>(g, F, W, pa, pb, tx, st);
}

}  // namespace

// Chunk length and x-tile width of the register sweeps for a line of n
// unknowns.  P is a power of two (2P <= 32 lets the reduced systems use warp
// PCR): the smallest with chunks of at most 16, else 16 chunks while they
// stay <= 32, else 32 chunks (reduced systems by Thomas); at most 1024
// threads per block for chunks <= 16, 512 above.
void sweep_geometry(int n, int &chunk, int &P, int &tx) {
    P = 1;
    while (P < 16 && (n + P - 1) / P > 16) P *= 2;
    if ((n + P - 1) / P > 32) P = 32;
    while (P > 1 && n / P < 3) P /= 2;
    chunk = (n + P - 1) / P;
    const int maxthr = chunk <= 16 ? 256 : 512;
    tx = 32;
    while (tx > 1 && tx * P > maxthr) tx /= 2;
}

// Chunks per line and x columns per block of the uniform y sweep: P the
// smallest power of two giving chunks of at most 16 (at most 32 chunks, so a
// line's carries fit one warp); up to 32 columns in a block of at most 256
// threads.
void sweep_y_geometry(int n, int &chunk, int &P, int &tx) {
    P = 1;
    while (P < 32 && (n + P - 1) / P > 16) P *= 2;
    chunk = (n + P - 1) / P;
    tx = 256 / P < 32 ? 256 / P : 32;
}

template <typename T, int L>
void launch_y_uni(const GridDev &g, Work<T> &W, const StepScalars *sc, cudaStream_t st) {
    const int tx = W.tx_y, P = W.py;
    const int nxt = (g.nx + tx - 1) / tx;
    const int threads = ((tx * P + 31) / 32) * 32;
    const size_t sm = 2 * sizeof(T) * tx * P;
    if (g.ny == L * P)
        K_sweep_y_uni<T, L, true>.launch(W.pdl != 0, dim3(3 * g.nz * nxt), dim3(threads), sm, st, g,
                                         W.q0, W.q1, W.q2, sc, P, tx);
    else
        K_sweep_y_uni<T, L, false>.launch(W.pdl != 0, dim3(3 * g.nz * nxt), dim3(threads), sm, st,
                                          g, W.q0, W.q1, W.q2, sc, P, tx);
}

template <typename T> void launch_sweep_y(const GridDev &g, Work<T> &W, const StepScalars *sc,
                                          cudaStream_t st) {
    if (W.chunk_y <= 8) launch_y_uni<T, 8>(g, W, sc, st);
    else if (W.chunk_y == 12) launch_y_uni<T, 12>(g, W, sc, st);
    else if (W.chunk_y <= 16) launch_y_uni<T, 16>(g, W, sc, st);
    else launch_y_uni<T, 32>(g, W, sc, st);
}

template <typename T> void launch_sweep_z(const GridDev &g, const Fields<T> &F, Work<T> &W,
                                          cudaStream_t st) {
    dispatch<T, 2, 0>(g, F, W, st);
}

template <typename T> void launch_sweep_z_adjoint(const GridDev &g, Work<T> &W, cudaStream_t st) {
    Fields<T> none;
    memset(&none, 0, sizeof none);
    dispatch<T, 2, 1>(g, none, W, st);
}

template <typename T> void set_smem_limits_lines(const GridDev &g, const Work<T> &W) {
    (void)g;
    (void)W;
    raise_smem_limit(K_sweep_y_uni<T, 8, false>.solo());
    raise_smem_limit(K_sweep_y_uni<T, 8, true>.solo());
    raise_smem_limit(K_sweep_y_uni<T, 12, false>.solo());
    raise_smem_limit(K_sweep_y_uni<T, 12, true>.solo());
    raise_smem_limit(K_sweep_y_uni<T, 16, false>.solo());
    raise_smem_limit(K_sweep_y_uni<T, 16, true>.solo());
    raise_smem_limit(K_sweep_y_uni<T, 32, false>.solo());
    raise_smem_limit(K_sweep_y_uni<T, 32, true>.solo());
    raise_smem_limit(K_sweep_reg<T, 8, 2, 0>.solo());
    raise_smem_limit(K_sweep_reg<T, 12, 2, 0>.solo());
    raise_smem_limit(K_sweep_reg<T, 24, 2, 0>.solo());
    raise_smem_limit(K_sweep_reg<T, 12, 2, 1>.solo());
    raise_smem_limit(K_sweep_reg<T, 24, 2, 1>.solo());
    raise_smem_limit(K_sweep_reg<T, 16, 2, 0>.solo());
    raise_smem_limit(K_sweep_reg<T, 32, 2, 0>.solo());
    raise_smem_limit(K_sweep_reg<T, 8, 2, 1>.solo());
    raise_smem_limit(K_sweep_reg<T, 16, 2, 1>.solo());
    raise_smem_limit(K_sweep_reg<T, 32, 2, 1>.solo());
    raise_smem_limit(K_sweep_reg<T, 8, 2, 0, 2>.solo());
    raise_smem_limit(K_sweep_reg<T, 12, 2, 0, 2>.solo());
    raise_smem_limit(K_sweep_reg<T, 16, 2, 0, 2>.solo());
    raise_smem_limit(K_sweep_reg<T, 8, 2, 1, 2>.solo());
    raise_smem_limit(K_sweep_reg<T, 12, 2, 1, 2>.solo());
    raise_smem_limit(K_sweep_reg<T, 16, 2, 1, 2>.solo());
}

#define FSEI_INST(T)                                                                           \
    template void launch_sweep_y<T>(const GridDev &, Work<T> &, const StepScalars *,           \
                                    cudaStream_t);                                            \
    template void launch_sweep_z<T>(const GridDev &, const Fields<T> &, Work<T> &,             \
                                    cudaStream_t);                                            \
    template void launch_sweep_z_adjoint<T>(const GridDev &, Work<T> &, cudaStream_t);         \
    template void set_smem_limits_lines<T>(const GridDev &, const Work<T> &);
FSEI_INST(float)
FSEI_INST(double)
#undef FSEI_INST

}  // namespace fsei
