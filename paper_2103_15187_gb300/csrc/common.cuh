// Internal definitions shared by the kernels and the host library of
// libfsei.so (fractional-step Navier-Stokes step, arXiv 2103.15187 Sec. 2.1,
// Sec. 3.1).  Nothing here is part of the public ABI (include/fsei.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define FSEI_HD __host__ __device__ __forceinline__
#define FSEI_D __device__ __forceinline__

// Programmatic dependent launch (griddepcontrol): a kernel launched with the
// programmatic-serialisation attribute may be scheduled while the previous
// kernel of its stream finishes.  pdl_wait() blocks until that kernel has
// completed and its memory operations are visible (a no-op for an ordinary
// launch); the hot kernels call it before any global memory access.
// pdl_trigger() allows the next such kernel to be scheduled once every block
// of this one has called it.
FSEI_D void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
FSEI_D void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

namespace fsei {

// ----------------------------------------------------------- complex -------
template <typename T> struct cplx { T re, im; };
template <typename T> struct alignas(2 * sizeof(T)) cplxa { T re, im; };

template <typename T> FSEI_HD cplx<T> cmk(T a, T b) { return {a, b}; }
template <typename T> FSEI_HD cplx<T> operator+(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> FSEI_HD cplx<T> operator-(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> FSEI_HD cplx<T> operator*(cplx<T> a, cplx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> FSEI_HD cplx<T> operator*(T s, cplx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> FSEI_HD cplx<T> conj(cplx<T> a) { return {a.re, -a.im}; }
// multiply by -i (sign < 0) or +i (sign > 0)
template <typename T, int SIGN> FSEI_HD cplx<T> mul_i(cplx<T> a) {
    return SIGN < 0 ? cplx<T>{a.im, -a.re} : cplx<T>{-a.im, a.re};
}

// -------------------------------------------------------------- grid -------
// Mesh description on the device.  z metrics are kept in double and float;
// kernels pick the copy matching their arithmetic type.
struct GridDev {
    int nx, ny, nz;
    int walls;          // 1: no-slip walls in z, 0: periodic z
    int mx;             // nx / 2 (length of the half-size complex x FFT)
    int sk;             // row stride (complex elements) of the spectrum
    double dx, dy, idx, idy, idx2, idy2;
    const double *dz, *idz, *ihc;   // dz[nz], 1/dz[nz], 1/hc[nz+1]
    const double *zf;               // the z faces z_0 .. z_nz (nz + 1; NULL
                                    // where no kernel needs them)
    const float *dzf, *idzf, *ihcf;
    // float roundings of dx, dy, idx, idy, idx2, idy2 and dx dy (the
    // single-precision kernels read these rather than convert per thread:
    // GB300's double-precision pipe is narrow)
    float fdx, fdy, fidx, fidy, fidx2, fidy2, fvxy;
};

// Set the float copies of a GridDev's double x/y spacings.
inline void grid_float_copies(GridDev &g) {
    g.fdx = (float)g.dx; g.fdy = (float)g.dy;
    g.fidx = (float)g.idx; g.fidy = (float)g.idy;
    g.fidx2 = (float)g.idx2; g.fidy2 = (float)g.idy2;
    g.fvxy = (float)(g.dx * g.dy);
}

// The double (T = double) or float (T = float) copy of a scalar kept in
// both precisions.
template <typename T> FSEI_HD T fpick(double d, float f);
template <> FSEI_HD double fpick<double>(double d, float) { return d; }
template <> FSEI_HD float fpick<float>(double, float f) { return f; }

template <typename T> struct Metric;
template <> struct Metric<double> {
    static FSEI_D const double *idz(const GridDev &g) { return g.idz; }
    static FSEI_D const double *ihc(const GridDev &g) { return g.ihc; }
    static FSEI_D const double *dz(const GridDev &g) { return g.dz; }
};
template <> struct Metric<float> {
    static FSEI_D const float *idz(const GridDev &g) { return g.idzf; }
    static FSEI_D const float *ihc(const GridDev &g) { return g.ihcf; }
    static FSEI_D const float *dz(const GridDev &g) { return g.dzf; }
};

// ---------------------------------------------------- per-step scalars -----
// Device-resident scalars of the running step (written by k_step_begin and
// the reductions; read by every kernel so that dt computed from the CFL
// condition never visits the host).
struct StepScalars {
    double dt;            // this fractional step's dt (alpha dt_n)
    double dt_step;       // dt_n of the full time step (equal to dt unless
                          // the step is split into Runge-Kutta sub-steps)
    double beta;          // dt / (2 Re)
    double gamma, rho;    // Adams-Bashforth weights of this step
    unsigned long long speed_cur;   // bits of max(|u_c|/dx+...) of u^n
    unsigned long long speed_next;  // same, accumulated for u^{n+1}
    unsigned long long maxdiv;      // bits of max |D u^{n+1}|
    double ke;            // kinetic energy of u^{n+1}
    int flags;            // FSEI_FLAG_*
    int pad;
    // factors of the uniform periodic x and y sweep matrices (tri.cuh,
    // uni_solve): alpha and 1/c for r = beta/dx^2 and beta/dy^2
    double ax, cix, ay, ciy;
    double invdt;         // 1 / dt
    // float roundings of dt, beta, gamma, rho, 1/dt and the four factors
    // above, for the single-precision kernels
    float fdt, fbeta, fgamma, frho, finvdt, fax, fcix, fay, fciy;
    // decay length of the x factor: the least n with |alpha_x|^n <= 2^-32
    // (single precision) and <= 2^-62 (double); the carry of an x line
    // across more unknowns than that is below the precision's rounding
    int ndecx_f, ndecx_d;
};

// --------------------------------------------- partitioned tridiagonal -----
// A line of n unknowns is cut into P chunks [s_p, e_p], s_p = p n / P.
// Chunk interiors are eliminated independently (each interior unknown is
// expressed through the two chunk ends), the 2P chunk ends form a reduced
// tridiagonal system (cyclic when the line is periodic), solved per line,
// and the interiors are recovered by one backward pass.  The matrix-only
// factors are the same for every line of a sweep; they are built once per
// step on the device (k_step_begin) into a TriPlan.
template <typename T> struct TriPlan {
    int n, P, cyclic, off;   // off: first unknown's index in the stored line
    int pad;                 // 1: unknown n-1 is a decoupled identity row past
                             // the stored line (never loaded or stored), which
                             // makes n a multiple of the chunk length
    const T *a, *c;          // sub- and super-diagonal (n)
    const T *inv;            // interior forward pivots 1/den_i (n)
    const T *at, *ct;        // interior forward factors a~_i, c~_i (n)
    const T *rlo, *rinv, *rcp, *rz; // reduced system (2P): couplings and LU
    const T *rsc;            // [0] = a_0/g (cyclic), [1] = 1/(1+v.z)
    // Parallel cyclic reduction of the reduced system (when 2P is a power of
    // two <= 128): level l combines equation i with i -/+ 2^l through the
    // multipliers pk1, pk2 [l * 2P + i]; pdinv are the final reciprocal
    // diagonals.  levels = 0 selects the Thomas path above.
    int levels;
    const T *pk1, *pk2, *pdinv;
};

// Levels of parallel cyclic reduction a plan stores multipliers for (2P <=
// 2^kPcrLevels).
constexpr int kPcrLevels = 7;

// Raw (mutable) storage of one plan inside the workspace.
template <typename T> struct TriPlanStore {
    T *a, *c, *inv, *at, *ct, *rlo, *rinv, *rcp, *rz, *rsc;
    T *pk1, *pk2, *pdinv;
};

// p n < 2^31 for the line lengths and chunk counts used here (n <= 2048,
// P <= 64); P is usually a power of two (a shift)
FSEI_HD int chunk_start(int p, int n, int P) {
#ifdef __CUDA_ARCH__
    return (P & (P - 1)) == 0 ? (p * n) >> (31 - __clz(P)) : (p * n) / P;
#else
    return (p * n) / P;
#endif
}

// An opaque copy of a pointer: addresses formed from it are recomputed
// rather than kept live in registers from an earlier use of the original.
template <typename P> FSEI_D P *fresh(P *p) {
    asm volatile("" : "+l"(p));
    return p;
}

// x mod d and x / d for x >= 0, d > 0: shifts when d is a power of two (the
// usual transform and tile sizes), the integer division otherwise
FSEI_D int dmod(int x, int d) { return (d & (d - 1)) == 0 ? (x & (d - 1)) : x % d; }
FSEI_D int ddiv(int x, int d) { return (d & (d - 1)) == 0 ? (x >> (31 - __clz(d))) : x / d; }

// ------------------------------------------------ asynchronous copies ------
// cp.async: global -> shared copies that complete in the background (no
// register staging, so a thread can have all of its copies in flight).
// 16 (8, 4) bytes: both addresses 16 (8, 4)-byte aligned.
FSEI_D void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
FSEI_D void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
FSEI_D void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
// wait for every copy this thread has issued (a barrier must follow before
// other threads read them)
FSEI_D void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// close the group of copies issued since the last commit; wait until at
// most one of this thread's groups is still in flight (the ones before it
// have landed; visible to this thread without a barrier)
FSEI_D void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
FSEI_D void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Copy rows of row_bytes bytes (row r: gsrc + r gstride -> sdst + r sstride)
// with every thread of the block issuing copies.  16-byte copies when the
// row length, both strides and both bases are multiples of 16 bytes, 4-byte
// copies otherwise (then all of them must be multiples of 4).
FSEI_D void copy_rows_async(void *sdst, size_t sstride, const void *gsrc, size_t gstride,
                            int rows, int row_bytes) {
    unsigned char *sd = static_cast<unsigned char *>(sdst);
    const unsigned char *gs = static_cast<const unsigned char *>(gsrc);
    const bool v16 = ((row_bytes | sstride | gstride) & 15) == 0 &&
                     (((uintptr_t)sd | (uintptr_t)gs) & 15) == 0;
    const int w = v16 ? 16 : 4;
    const int per = row_bytes / w;
    const int total = rows * per;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int r = ddiv(e, per), c = (e - r * per) * w;
        if (v16) cp_async16(sd + r * sstride + c, gs + r * gstride + c);
        else cp_async4(sd + r * sstride + c, gs + r * gstride + c);
    }
}

// bit pattern of a non-negative double, monotone in its value
FSEI_D unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
FSEI_D double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }

}  // namespace fsei
