// Pressure-increment Poisson solve of the fractional step (Sec. 2.1: the
// elliptic equation enforcing mass conservation; Sec. 4: solved through
// the periodic x-y directions by Fourier transforms -- FFTW3 in the paper --
// and the wall-normal direction by tridiagonal systems).
//
//   k_rfft_x          s = D u* / dt (or a given field) at the cell centres,
//                     real-to-complex DFT along x (half-length complex FFT
//                     plus the even/odd split)
//   k_fft_y<SIGN>     complex DFT along y, forward or inverse
//   k_poisson_z       per mode (kx, ky): (L_z - lambda_x - lambda_y) phi = s
//                     along z (walls: Neumann rows; periodic z: cyclic),
//                     times 1/(nx ny)
//   k_poisson_exact   the (0, 0) mode (phi_0 pinned to 0, then the volume-
//                     weighted mean removed) and, in mixed precision, every
//                     near-zero mode, in double with Thomas' algorithm
//   k_irfft_x         complex-to-real inverse DFT along x into phi
#include <string.h>

#include "kernels.cuh"
#include "tri.cuh"

namespace fsei {

namespace {

// Row length (complex elements) of the x-transform lines in shared memory:
// mx rounded up to even, so that every line starts on a 16-byte boundary.
FSEI_HD int fft_x_ls(int mx) { return mx + (mx & 1); }
// Scratch row length of the x transforms (the two-pass transform's padded
// layout where it applies), even.
FSEI_HD int fft_x_bls(int mx) {
    const int b = fft_scratch_len(mx) > mx ? fft_scratch_len(mx) : mx;
    return b + (b & 1);
}
// complex values per staged spectrum row of the inverse x transform: kx <=
// mx, rounded up to whole 16-byte copies (within the row stride sk, a
// multiple of 16)
FSEI_HD int irfft_stage_row(int mx) { return (mx + 1 + 1) & ~1; }

// Stage the x twiddles w^m (m < mx) and the post-processing factors
// exp(-2 pi i kx / nx) (kx <= mx) in shared memory.
template <typename T>
FSEI_D void stage_x_twiddles(cplx<T> *TW, cplx<T> *TP, const cplx<T> *twx,
                             const cplx<T> *twpost, int mx) {
    for (int m = threadIdx.x; m < mx; m += blockDim.x) TW[m] = twx[m];
    for (int m = threadIdx.x; m <= mx; m += blockDim.x) TP[m] = twpost[m];
}

// Real-to-complex transform along x of RY rows (j0 .. j0+RY-1 of plane k):
// the real row of nx values is read as mx = nx/2 complex values (even
// entries real parts, odd entries imaginary parts), transformed with a
// half-length complex FFT, and split into the nx/2 + 1 coefficients
//   X_kx = (Z_kx + conj Z_{mx-kx}) / 2 - i w^kx (Z_kx - conj Z_{mx-kx}) / 2,
// w = exp(-2 pi i / nx).  MODE 0: the rows are s = D u* / dt, formed from
// the three velocity fields with every load of a thread in flight at once;
// MODE 1: the rows of a given field, copied asynchronously.
// Single precision: 4 blocks per SM (64 registers, no spills; 256^3: 80 ->
// 72 us against the compiler's 80 registers and 3 blocks).
template <typename T, int MODE, int RY>
FSEI_D void
k_rfft_x(GridDev g, const T *__restrict__ q0, const T *__restrict__ q1,
         const T *__restrict__ q2, const T *__restrict__ src, cplx<T> *__restrict__ spec,
         const cplx<T> *__restrict__ twx, const cplx<T> *__restrict__ twpost, FftPlanDev fp,
         const StepScalars *sc) {
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_wait();
    pdl_trigger();
    const int nx = g.nx, ny = g.ny, nz = g.nz, mx = g.mx, sk = g.sk;
    const int ls = fft_x_ls(mx);
    const int bls = fft_x_bls(mx);
    cplx<T> *A = reinterpret_cast<cplx<T> *>(smraw);
    cplx<T> *B = A + (size_t)RY * ls;
    cplx<T> *TW = B + (size_t)RY * bls;
    cplx<T> *TP = TW + fft_x_ls(mx);
    const int nby = ny / RY;
    const int k = blockIdx.x / nby, j0 = (blockIdx.x % nby) * RY;
    if (MODE == 1) {
        copy_rows_async(A, ls * sizeof(cplx<T>), src + ((size_t)k * ny + j0) * nx,
                        (size_t)nx * sizeof(T), RY, nx * (int)sizeof(T));
        stage_x_twiddles(TW, TP, twx, twpost, mx);
        cp_async_wait_all();
    } else {
        const T invdt = fpick<T>(sc->invdt, sc->finvdt);
        const bool hasup = !g.walls || k < nz - 1;
        const int ku = k == nz - 1 ? 0 : k + 1;
        const T idx = fpick<T>(g.idx, g.fidx), idy = fpick<T>(g.idy, g.fidy);
        const T idzk = Metric<T>::idz(g)[k];
        const int oc0 = (k * ny + j0) * nx, ou0 = (ku * ny + j0) * nx;
        constexpr int VW = 16 / (int)sizeof(T);
        struct alignas(16) V { T v[VW]; };
        if (nx % VW == 0) {
            // 16-byte vectors: VW consecutive cells of a row per item, the
            // u neighbour beyond the vector as a scalar
            const int nv = nx / VW;
#pragma unroll 4
            for (int e = threadIdx.x; e < RY * nv; e += blockDim.x) {
                const int r = ddiv(e, nv), i0 = (e - r * nv) * VW;
                const int o = oc0 + r * nx;
                const int ojp = (j0 + r == ny - 1) ? (k * ny) * nx : o + nx;
                const V a0 = *reinterpret_cast<const V *>(q0 + o + i0);
                const V a1 = *reinterpret_cast<const V *>(q1 + o + i0);
                const V a1p = *reinterpret_cast<const V *>(q1 + ojp + i0);
                const V a2 = *reinterpret_cast<const V *>(q2 + o + i0);
                V a2u;
                if (hasup) a2u = *reinterpret_cast<const V *>(q2 + ou0 + r * nx + i0);
                const T a0n = q0[o + (i0 + VW == nx ? 0 : i0 + VW)];
                V dv;
#pragma unroll
                for (int c = 0; c < VW; ++c) {
                    const T up = c == VW - 1 ? a0n : a0.v[c + 1];
                    const T wu = hasup ? a2u.v[c] : T(0);
                    dv.v[c] = ((up - a0.v[c]) * idx + (a1p.v[c] - a1.v[c]) * idy +
                               (wu - a2.v[c]) * idzk) * invdt;
                }
                *reinterpret_cast<V *>(reinterpret_cast<T *>(A + (size_t)r * ls) + i0) = dv;
            }
        } else
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const int ip = i == nx - 1 ? 0 : i + 1;
            T a0[RY], a0p[RY], a1[RY], a1p[RY], a2[RY], a2u[RY];
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                const int o = oc0 + r * nx;
                const int ojp = (j0 + r == ny - 1) ? (k * ny) * nx : o + nx;
                a0[r] = q0[o + i];
                a0p[r] = q0[o + ip];
                a1[r] = q1[o + i];
                a1p[r] = q1[ojp + i];
                a2[r] = q2[o + i];
                a2u[r] = hasup ? q2[ou0 + r * nx + i] : T(0);
            }
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                T *arow = reinterpret_cast<T *>(A + (size_t)r * ls);
                arow[i] = ((a0p[r] - a0[r]) * idx + (a1p[r] - a1[r]) * idy +
                           (a2u[r] - a2[r]) * idzk) * invdt;
            }
        }
        stage_x_twiddles(TW, TP, twx, twpost, mx);
    }
    __syncthreads();
    const cplx<T> *R = fft_lines_fast<T, -1, false>(A, B, 1, ls, bls, RY, fp, TW);
    const T hf = T(0.5);
    for (int e = threadIdx.x; e < RY * (mx + 1); e += blockDim.x) {
        const int r = e / (mx + 1), kx = e - r * (mx + 1);
        const cplx<T> zk = R[r * ls + (kx == mx ? 0 : kx)];
        const cplx<T> zc = conj(R[r * ls + (kx == 0 ? 0 : mx - kx)]);
        const cplx<T> ev = hf * (zk + zc);
        const cplx<T> od = mul_i<T, -1>(hf * (TP[kx] * (zk - zc)));
        spec[((size_t)k * ny + j0 + r) * sk + kx] = ev + od;
    }
}

// Complex DFT along y of tkx spectrum columns of plane k: the tile is
// copied asynchronously into shared memory (rows of tkx values), transformed
// with the line index fastest, and written back with 16-byte stores.
template <typename T, int SIGN>
FSEI_D void
k_fft_y(GridDev g, cplx<T> *__restrict__ spec, const cplx<T> *__restrict__ twy, FftPlanDev fp,
        int tkx) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int ny = g.ny, sk = g.sk;
    cplx<T> *A = reinterpret_cast<cplx<T> *>(smraw);
    cplx<T> *B = A + (size_t)ny * tkx;
    cplx<T> *TW = B + (size_t)ny * tkx;
    const int nkt = sk / tkx;
    const int k = blockIdx.x / nkt, x0 = (blockIdx.x % nkt) * tkx;
    cplx<T> *base = spec + (size_t)k * ny * sk + x0;
    const int rb = tkx * (int)sizeof(cplx<T>);
    copy_rows_async(A, rb, base, (size_t)sk * sizeof(cplx<T>), ny, rb);
    for (int m = threadIdx.x; m < ny; m += blockDim.x) TW[m] = twy[m];
    cp_async_wait_all();
    __syncthreads();
    const cplx<T> *R = fft_lines_fast<T, SIGN, true>(A, B, tkx, 1, 0, tkx, fp, TW);
    // 16-byte stores: rb is a multiple of 16 (tkx even in single precision)
    const int per = rb / 16;
    for (int e = threadIdx.x; e < ny * per; e += blockDim.x) {
        const int j = ddiv(e, per), c = e - j * per;
        const uint4 v = reinterpret_cast<const uint4 *>(R + (size_t)j * tkx)[c];
        reinterpret_cast<uint4 *>(base + (size_t)j * sk)[c] = v;
    }
}

// The y transform for power-of-two ny = N1 N2 <= 256 (fft_lines_2p's split)
// without staging tiles: pass 1 reads its N1 inputs per (line, n2) straight
// from the spectrum into registers (coalesced across the tkx kx columns of
// the block), applies the in-register DFT and the twiddles and writes the
// transposed values to shared memory; pass 2 reads them back, applies the
// second DFT and writes the result straight to the spectrum.  The block owns
// its tile, so reading and writing in place is safe.
template <typename T, int SIGN, int N1, int N2>
FSEI_D void
k_fft_y_2p(GridDev g, cplx<T> *__restrict__ spec, const cplx<T> *__restrict__ twy, int tkx) {
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_wait();
    pdl_trigger();
    constexpr int N = N1 * N2;
    const int sk = g.sk;
    cplx<T> *B = reinterpret_cast<cplx<T> *>(smraw);   // [N][tkx]
    cplx<T> *TW = B + (size_t)N * tkx;
    const int nkt = sk / tkx;
    const int k = blockIdx.x / nkt, x0 = (blockIdx.x % nkt) * tkx;
    cplx<T> *base = spec + (size_t)k * N * sk + x0;
    const int t = threadIdx.x;
    const int nt = (int)blockDim.x;
    // pass 1: (n2, line) pairs, in turn when there are more than threads
    auto pass1_load = [&](int task, cplx<T> (&x)[N1]) {
        const int m2 = ddiv(task, tkx), m1 = task - m2 * tkx;
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) x[n1] = base[(size_t)(n1 * N2 + m2) * sk + m1];
    };
    auto pass1_rest = [&](int task, cplx<T> (&x)[N1]) {
        const int m2 = ddiv(task, tkx), m1 = task - m2 * tkx;
        dft_reg<T, N1, SIGN>(x, TW, N);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) {
            cplx<T> w = TW[m2 * k1];
            if (SIGN > 0) w = conj(w);
            x[k1] = x[k1] * w;
        }
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) B[(m2 * N1 + k1) * tkx + m1] = x[k1];
    };
    const bool on1 = t < tkx * N2;
    cplx<T> x[N1];
    if (on1) pass1_load(t, x);
    for (int m = t; m < N; m += nt) TW[m] = twy[m];
    __syncthreads();
    if (on1) pass1_rest(t, x);
    for (int task = t + nt; task < tkx * N2; task += nt) {
        pass1_load(task, x);
        pass1_rest(task, x);
    }
    __syncthreads();
    for (int task = t; task < tkx * N1; task += nt) {
        const int k1 = ddiv(task, tkx), l2 = task - k1 * tkx;
        cplx<T> y[N2];
#pragma unroll
        for (int q = 0; q < N2; ++q) y[q] = B[(q * N1 + k1) * tkx + l2];
        dft_reg<T, N2, SIGN>(y, TW, N);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) base[(size_t)(k1 + N1 * k2) * sk + l2] = y[k2];
    }
}

// z operator of the modes in a block; a, c and -(a + c) staged in shared
// memory (a(0) and c(nz-1) are the periodic couplings, 0 with walls)
template <typename T> struct PoissonMat {
    const T *sa, *sc, *sb0, *lam;
    FSEI_D T a(int i) const { return sa[i]; }
    FSEI_D T c(int i) const { return sc[i]; }
    FSEI_D T b(int l, int i) const { return sb0[i] - lam[l]; }
};

template <typename T>
FSEI_D void
k_poisson_z(GridDev g, cplx<T> *__restrict__ spec, const T *__restrict__ lamx,
            const T *__restrict__ lamy, const unsigned char *__restrict__ exact, int tkx, int P,
            T scale) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int ny = g.ny, nz = g.nz, sk = g.sk;
    const int rs = 2 * P + 1;
    cplx<T> *D = reinterpret_cast<cplx<T> *>(smraw);
    cplx<T> *rr = D + (size_t)nz * tkx;
    T *fa = reinterpret_cast<T *>(rr + (size_t)tkx * rs);
    T *fc = fa + (size_t)nz * tkx;
    T *rlo = fc + (size_t)nz * tkx;
    T *rdi = rlo + (size_t)tkx * rs;
    T *rup = rdi + (size_t)tkx * rs;
    T *lam = rup + (size_t)tkx * rs;
    T *sa = lam + tkx, *scc = sa + nz, *sb0 = scc + nz;
    const int nkt = sk / tkx;
    const int ky = blockIdx.x / nkt, x0 = (blockIdx.x % nkt) * tkx;
    if (threadIdx.x < tkx) {
        T lv = lamx[x0 + threadIdx.x] + lamy[ky];
        // the singular (0, 0) mode is solved by k_poisson_exact; keep this
        // (discarded) copy of its system regular
        if (x0 + threadIdx.x == 0 && ky == 0) lv = T(1);
        lam[threadIdx.x] = lv;
    }
    const size_t plane = (size_t)ny * sk;
    cplx<T> *base = spec + (size_t)ky * sk + x0;
    copy_rows_async(D, tkx * sizeof(cplx<T>), base, plane * sizeof(cplx<T>), nz,
                    tkx * (int)sizeof(cplx<T>));
    {
        const T *idz = Metric<T>::idz(g), *ihc = Metric<T>::ihc(g);
        for (int k = threadIdx.x; k < nz; k += blockDim.x) {
            const T a = (g.walls && k == 0) ? T(0) : ihc[k] * idz[k];
            const T c = (g.walls && k == nz - 1) ? T(0) : ihc[k + 1] * idz[k];
            sa[k] = a;
            scc[k] = c;
            sb0[k] = -(a + c);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    PoissonMat<T> M{sa, scc, sb0, lam};
    tri_fly_solve<T>(D, tkx, 1, fa, fc, tkx, 1, tkx, nz, P, !g.walls, M, rr, rlo, rdi, rup, rs);
    // modes solved exactly in double (k_poisson_exact, launched before this
    // kernel) keep their values
    const unsigned char *ex = exact + (size_t)ky * sk + x0;
    for (int e = threadIdx.x; e < nz * tkx; e += blockDim.x) {
        const int k = e / tkx, l = e - k * tkx;
        if (!ex[l]) base[(size_t)k * plane + l] = scale * D[e];
    }
}

// z operator of one exactly solved mode in double: rows k = i + shift of the
// line (shift 1 for the pinned (0, 0) mode, whose unknown at k = 0 is fixed
// to 0; its neighbours at k = 0 and, with periodic z, k = nz are then
// Dirichlet zeros and drop out of the first and last rows).
struct ExactMat {
    const double *idz, *ihc;
    double lam;
    int nz, walls, shift;
    FSEI_D double acut(int k) const { return (walls && k == 0) ? 0.0 : ihc[k] * idz[k]; }
    FSEI_D double ccut(int k) const { return (walls && k == nz - 1) ? 0.0 : ihc[k + 1] * idz[k]; }
    FSEI_D double a(int i) const { return acut(i + shift); }
    FSEI_D double c(int i) const { return ccut(i + shift); }
    FSEI_D double b(int, int i) const { return -(acut(i + shift) + ccut(i + shift)) - lam; }
};

// One block per exactly solved mode: the z line is staged in shared memory
// in double and solved with the partitioned elimination of tri.cuh (chunks
// in parallel, reduced system on one thread), then written back scaled by
// 1/(nx ny).  For the (0, 0) mode the volume-weighted mean is removed
// afterwards (gauge); with compat its right-hand side first loses its own
// dz-weighted mean (makes an arbitrary right-hand side compatible).
template <typename T>
FSEI_D void
k_poisson_exact(GridDev g, cplx<T> *spec, const int *modes, const double *lamx,
                const double *lamy, double scale, int compat, int P) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nz = g.nz;
    const int rs = 2 * P + 1;
    cplx<double> *D = reinterpret_cast<cplx<double> *>(smraw);
    cplx<double> *rr = D + nz;
    double *fa = reinterpret_cast<double *>(rr + rs);
    double *fc = fa + nz, *rlo = fc + nz, *rdi = rlo + rs, *rup = rdi + rs;
    __shared__ double red[2][64];
    const int code = modes[blockIdx.x];
    const int kx = code % g.sk, ky = code / g.sk;
    const bool zero_mode = kx == 0 && ky == 0;
    const size_t stride = (size_t)g.ny * g.sk;
    cplx<T> *line = spec + (size_t)ky * g.sk + kx;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        const cplx<T> v = line[(size_t)k * stride];
        D[k] = cplx<double>{(double)v.re, (double)v.im};
    }
    __syncthreads();
    auto wmean = [&](double &mr, double &mi) {
        double sr = 0.0, si = 0.0;
        for (int k = threadIdx.x; k < nz; k += blockDim.x) {
            sr += D[k].re * g.dz[k];
            si += D[k].im * g.dz[k];
        }
        red[0][threadIdx.x] = sr;
        red[1][threadIdx.x] = si;
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0, w = 0.0;
            for (int t = 0; t < (int)blockDim.x; ++t) { a += red[0][t]; b += red[1][t]; }
            for (int k = 0; k < nz; ++k) w += g.dz[k];
            red[0][0] = a / w;
            red[1][0] = b / w;
        }
        __syncthreads();
        mr = red[0][0];
        mi = red[1][0];
        __syncthreads();
    };
    if (zero_mode && compat) {
        double mr, mi;
        wmean(mr, mi);
        for (int k = threadIdx.x; k < nz; k += blockDim.x) { D[k].re -= mr; D[k].im -= mi; }
        __syncthreads();
    }
    ExactMat M{g.idz, g.ihc, lamx[kx] + lamy[ky], nz, g.walls, zero_mode ? 1 : 0};
    const int n = zero_mode ? nz - 1 : nz;
    int Pl = P;
    if (Pl > n / 3) Pl = n / 3;
    if (Pl < 1) Pl = 1;
    tri_fly_solve<double>(D + M.shift, 1, 0, fa, fc, 1, 0, 1, n, Pl, (!g.walls && !zero_mode), M,
                          rr, rlo, rdi, rup, rs);
    if (zero_mode && threadIdx.x == 0) D[0] = cplx<double>{0.0, 0.0};
    __syncthreads();
    double mr = 0.0, mi = 0.0;
    if (zero_mode) wmean(mr, mi);
    for (int k = threadIdx.x; k < nz; k += blockDim.x)
        line[(size_t)k * stride] = cplx<T>{T((D[k].re - mr) * scale), T((D[k].im - mi) * scale)};
}

// Exactly solved modes with factors computed at grid creation: one warp
// per mode solves, in double, the forward recurrence y_i = xa_i y_{i-1} +
// xm_i s_i and the backward one phi_i = y_i - xc_i phi_{i+1} (Thomas'
// algorithm) as parallel scans of affine maps: lane l composes the maps of
// its E consecutive rows, a shuffle scan over the lanes gives each lane its
// incoming value, and the lane re-runs its rows from it.  Cyclic lines (a
// non-zero mode with periodic z) add the Sherman-Morrison correction phi -=
// xz (v . y) / (1 + v . z), v . y = y_0 + v_last y_{n-1}.  The (0, 0) mode
// pins phi_0 = 0 (rows 1 .. nz-1) and removes the volume-weighted mean, as
// k_poisson_exact does.
// One warp (lane = 0 .. 31) solves exactly solved mode number `mode`; D:
// shared scratch of nz values.
template <typename T>
__device__ __forceinline__ void exact_mode_solve(const GridDev &g, cplx<T> *spec, int mode,
                                                 const int *modes, const double *xa,
                                                 const double *xm, const double *xc,
                                                 const double *xz, const double *xs,
                                                 double scale, int compat, double zlen,
                                                 cplx<double> *D, int lane) {
    const int nz = g.nz;
    const int code = modes[mode];
    const int kx = code % g.sk, ky = code / g.sk;
    const bool zero_mode = kx == 0 && ky == 0;
    const bool cyclic = !g.walls && !zero_mode;
    const size_t stride = (size_t)g.ny * g.sk;
    cplx<T> *line = spec + (size_t)ky * g.sk + kx;
    for (int k = lane; k < nz; k += 32) {
        const cplx<T> v = line[(size_t)k * stride];
        D[k] = cplx<double>{(double)v.re, (double)v.im};
    }
    __syncwarp();
    // dz-weighted mean of the line (warp reduction)
    auto wmean = [&](double &mr, double &mi) {
        double sr = 0.0, si = 0.0;
        for (int k = lane; k < nz; k += 32) {
            sr += D[k].re * g.dz[k];
            si += D[k].im * g.dz[k];
        }
        for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
            si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        mr = sr / zlen;
        mi = si / zlen;
    };
    if (zero_mode && compat) {
        double mr, mi;
        wmean(mr, mi);
        __syncwarp();
        for (int k = lane; k < nz; k += 32) { D[k].re -= mr; D[k].im -= mi; }
        __syncwarp();
    }
    const int shift = zero_mode ? 1 : 0, n = nz - shift;
    cplx<double> *d = D + shift;
    const size_t o = (size_t)mode * nz;
    const double *A = xa + o, *M = xm + o, *C = xc + o;
    const int E = (n + 31) / 32;
    const int i0 = lane * E < n ? lane * E : n, i1 = i0 + E < n ? i0 + E : n;
    // forward: y_i = A_i y_{i-1} + M_i s_i
    {
        double ga = 1.0, gr = 0.0, gi = 0.0;
        for (int i = i0; i < i1; ++i) {
            ga = A[i] * ga;
            gr = A[i] * gr + M[i] * d[i].re;
            gi = A[i] * gi + M[i] * d[i].im;
        }
        for (int s = 1; s < 32; s <<= 1) {
            const double pa = __shfl_up_sync(0xffffffffu, ga, s);
            const double pr = __shfl_up_sync(0xffffffffu, gr, s);
            const double pi = __shfl_up_sync(0xffffffffu, gi, s);
            if (lane >= s) {
                gr = ga * pr + gr;
                gi = ga * pi + gi;
                ga = ga * pa;
            }
        }
        double yr = __shfl_up_sync(0xffffffffu, gr, 1), yi = __shfl_up_sync(0xffffffffu, gi, 1);
        if (lane == 0) yr = yi = 0.0;
        for (int i = i0; i < i1; ++i) {
            yr = A[i] * yr + M[i] * d[i].re;
            yi = A[i] * yi + M[i] * d[i].im;
            d[i] = cplx<double>{yr, yi};
        }
    }
    __syncwarp();
    // backward: phi_i = y_i - C_i phi_{i+1}
    {
        double ga = 1.0, gr = 0.0, gi = 0.0;
        for (int i = i1 - 1; i >= i0; --i) {
            ga = -C[i] * ga;
            gr = d[i].re - C[i] * gr;
            gi = d[i].im - C[i] * gi;
        }
        for (int s = 1; s < 32; s <<= 1) {
            const double pa = __shfl_down_sync(0xffffffffu, ga, s);
            const double pr = __shfl_down_sync(0xffffffffu, gr, s);
            const double pi = __shfl_down_sync(0xffffffffu, gi, s);
            if (lane + s < 32) {
                gr = ga * pr + gr;
                gi = ga * pi + gi;
                ga = ga * pa;
            }
        }
        double xr = __shfl_down_sync(0xffffffffu, gr, 1), xi = __shfl_down_sync(0xffffffffu, gi, 1);
        if (lane == 31) xr = xi = 0.0;
        for (int i = i1 - 1; i >= i0; --i) {
            xr = d[i].re - C[i] * xr;
            xi = d[i].im - C[i] * xi;
            d[i] = cplx<double>{xr, xi};
        }
    }
    __syncwarp();
    if (cyclic) {
        const double vl = xs[2 * mode], fac = xs[2 * mode + 1];
        const double sr = fac * (d[0].re + vl * d[n - 1].re);
        const double si = fac * (d[0].im + vl * d[n - 1].im);
        __syncwarp();
        const double *Z = xz + o;
        for (int i = lane; i < n; i += 32) {
            d[i].re -= Z[i] * sr;
            d[i].im -= Z[i] * si;
        }
        __syncwarp();
    }
    double mr = 0.0, mi = 0.0;
    if (zero_mode) {
        if (lane == 0) D[0] = cplx<double>{0.0, 0.0};
        __syncwarp();
        wmean(mr, mi);
    }
    for (int k = lane; k < nz; k += 32)
        line[(size_t)k * stride] = cplx<T>{T((D[k].re - mr) * scale), T((D[k].im - mi) * scale)};
}

template <typename T>
FSEI_D void
k_poisson_exact_f(GridDev g, cplx<T> *spec, const int *modes, const double *xa,
                  const double *xm, const double *xc, const double *xz, const double *xs,
                  double scale, int compat, double zlen) {
    extern __shared__ __align__(16) unsigned char smraw[];
    exact_mode_solve<T>(g, spec, blockIdx.x, modes, xa, xm, xc, xz, xs, scale, compat, zlen,
                        reinterpret_cast<cplx<double> *>(smraw), threadIdx.x);
}

// Lane-resident z solve: one warp segment of LPL lanes per Fourier mode
// line (kx, ky), lane r holding rows r E .. r E + E - 1 (nz = LPL E) of
// (L_z - lambda_x - lambda_y) phi = s in registers.  The block owns NL =
// 256 / LPL consecutive kx columns of one ky row; the tile is staged in
// shared memory by asynchronous copies, XOR-swizzled so that the lanes'
// strided rows fall in different banks.  Each lane eliminates its chunk
// interior with factors formed on the fly (as tri_fly_solve), which leaves
// two unknowns per lane (its first and last row) in a tridiagonal system of
// 2 LPL unknowns coupled cyclically across the lanes (with walls the end
// couplings are zero, so the cyclic indexing changes nothing); parallel
// cyclic reduction over lane shuffles solves it in log2(2 LPL) levels, and
// each lane substitutes back into its chunk.  Blocks 0 .. n_exact-1 instead
// solve the exactly handled modes in double (exact_mode_solve), starting
// before the others; the other blocks read those modes but do not store
// them.  Results scaled by 1/(nx ny).
template <typename T> struct alignas(4 * sizeof(T)) ZCoef { T a, c, b0, pad; };

// Single precision: 3 blocks per SM (80 registers; 256^3: 47 -> 44 us
// against 117 registers and 2 blocks).
template <typename T, int E, int LPL>
FSEI_D void
k_poisson_zl(GridDev g, cplx<T> *__restrict__ spec, const T *__restrict__ lamx,
             const T *__restrict__ lamy, const unsigned char *__restrict__ exact, T scale,
             int n_exact, const int *modes, const double *xa, const double *xm,
             const double *xc, const double *xz, const double *xs, double dscale, int compat,
             double zlen) {
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_wait();
    pdl_trigger();
    if ((int)blockIdx.x < n_exact) {
        if (threadIdx.x < 32)
            exact_mode_solve<T>(g, spec, blockIdx.x, modes, xa, xm, xc, xz, xs, dscale, compat,
                                zlen, reinterpret_cast<cplx<double> *>(smraw), threadIdx.x);
        return;
    }
    constexpr int NL = 256 / LPL;                                // lines per block
    constexpr int SLOTS = 128 / (2 * (int)sizeof(T));            // values per 128 bytes
    constexpr int GR = SLOTS > NL ? SLOTS / NL : 1;              // tile rows per group
    constexpr int GW = GR * NL;
    static_assert(E % GR == 0 && E >= 4, "chunk rows");
    const int nz = g.nz, ny = g.ny, sk = g.sk;
    cplx<T> *S = reinterpret_cast<cplx<T> *>(smraw);
    ZCoef<T> *C = reinterpret_cast<ZCoef<T> *>(S + (size_t)nz * NL);
    // tile position of value (z, line w): groups of GR rows, the values of a
    // group permuted by the lane index z / E of the reading lane
    auto pos = [](int z, int w) {
        return (z / GR) * GW + (((z % GR) * NL + w) ^ ((z / E) & (GW - 1)));
    };
    const int bl = blockIdx.x - n_exact;
    const int nkt = sk / NL;
    const int ky = bl / nkt, x0 = (bl - ky * nkt) * NL;
    const size_t plane = (size_t)ny * sk;
    const int t = threadIdx.x;
    cplx<T> *col = spec + (size_t)ky * sk + x0;
    for (int e = t; e < nz * NL; e += 256) {
        const int z = e / NL, w = e - z * NL;
        if (sizeof(T) == 4) cp_async8(S + pos(z, w), col + (size_t)z * plane + w);
        else cp_async16(S + pos(z, w), col + (size_t)z * plane + w);
    }
    {
        const T *idz = Metric<T>::idz(g), *ihc = Metric<T>::ihc(g);
        for (int k = t; k < nz; k += 256) {
            const T a = (g.walls && k == 0) ? T(0) : ihc[k] * idz[k];
            const T c = (g.walls && k == nz - 1) ? T(0) : ihc[k + 1] * idz[k];
            ZCoef<T> zc;
            zc.a = a;
            zc.c = c;
            zc.b0 = -(a + c);
            zc.pad = T(0);
            C[k + k / E] = zc;
        }
    }
    cp_async_wait_all();
    __syncthreads();
    const int lane = t & 31;
    const int r = lane & (LPL - 1);
    const int w = (t >> 5) * (32 / LPL) + lane / LPL;
    T lam = lamx[x0 + w] + lamy[ky];
    // the singular (0, 0) mode is solved in double; keep this (discarded)
    // copy of its system regular
    if (x0 + w == 0 && ky == 0) lam = T(1);
    const int s0 = r * E;
    const ZCoef<T> *cr = C + s0 + r;       // row s0 + i at cr[i]
    cplx<T> d[E];
#pragma unroll
    for (int i = 0; i < E; ++i) d[i] = S[pos(s0 + i, w)];
    // chunk interior: x_i = d~_i - a~_i x_s0 - c~_i x_{i+1}
    T at[E], ct[E];
    {
        const ZCoef<T> q = cr[1];
        const T inv = rcp(q.b0 - lam);
        at[1] = q.a * inv;
        ct[1] = q.c * inv;
        d[1] = cplx<T>{d[1].re * inv, d[1].im * inv};
    }
#pragma unroll
    for (int i = 2; i < E - 1; ++i) {
        const ZCoef<T> q = cr[i];
        const T inv = rcp((q.b0 - lam) - q.a * ct[i - 1]);
        at[i] = -q.a * at[i - 1] * inv;
        ct[i] = q.c * inv;
        d[i] = cplx<T>{(d[i].re - q.a * d[i - 1].re) * inv, (d[i].im - q.a * d[i - 1].im) * inv};
    }
    // x_{s0+1} through the chunk ends
    cplx<T> dh = d[E - 2];
    T ah = at[E - 2], ch = ct[E - 2];
#pragma unroll
    for (int i = E - 3; i >= 1; --i) {
        dh = cplx<T>{d[i].re - ct[i] * dh.re, d[i].im - ct[i] * dh.im};
        ah = at[i] - ct[i] * ah;
        ch = -ct[i] * ch;
    }
    // reduced rows: F (row s0) and E (row s0 + E - 1); L couples to the
    // unknown before, U to the one after in the order F_0 E_0 F_1 E_1 ...
    T Lf, Df, Uf, Le, De, Ue;
    cplx<T> Rf, Re;
    {
        const ZCoef<T> q = cr[0];
        Lf = q.a;
        Df = (q.b0 - lam) - q.c * ah;
        Uf = -q.c * ch;
        Rf = cplx<T>{d[0].re - q.c * dh.re, d[0].im - q.c * dh.im};
        const ZCoef<T> u = cr[E - 1];
        Le = -u.a * at[E - 2];
        De = (u.b0 - lam) - u.a * ct[E - 2];
        Ue = u.c;
        Re = cplx<T>{d[E - 1].re - u.a * d[E - 2].re, d[E - 1].im - u.a * d[E - 2].im};
    }
    // parallel cyclic reduction; stride 1 couples F_r with E_{r-1} and E_r,
    // E_r with F_r and F_{r+1}
    {
        const int rm = (r - 1) & (LPL - 1), rp = (r + 1) & (LPL - 1);
        const T pLe = __shfl_sync(0xffffffffu, Le, rm, LPL);
        const T pDe = __shfl_sync(0xffffffffu, De, rm, LPL);
        const T pUe = __shfl_sync(0xffffffffu, Ue, rm, LPL);
        const T pRer = __shfl_sync(0xffffffffu, Re.re, rm, LPL);
        const T pRei = __shfl_sync(0xffffffffu, Re.im, rm, LPL);
        const T nLf = __shfl_sync(0xffffffffu, Lf, rp, LPL);
        const T nDf = __shfl_sync(0xffffffffu, Df, rp, LPL);
        const T nUf = __shfl_sync(0xffffffffu, Uf, rp, LPL);
        const T nRfr = __shfl_sync(0xffffffffu, Rf.re, rp, LPL);
        const T nRfi = __shfl_sync(0xffffffffu, Rf.im, rp, LPL);
        const T f1 = -Lf * rcp(pDe), f2 = -Uf * rcp(De);
        const T e1 = -Le * rcp(Df), e2 = -Ue * rcp(nDf);
        const T Lf2 = f1 * pLe, Uf2 = f2 * Ue, Df2 = Df + f1 * pUe + f2 * Le;
        const cplx<T> Rf2{Rf.re + f1 * pRer + f2 * Re.re, Rf.im + f1 * pRei + f2 * Re.im};
        const T Le2 = e1 * Lf, Ue2 = e2 * nUf, De2 = De + e1 * Uf + e2 * nLf;
        const cplx<T> Re2{Re.re + e1 * Rf.re + e2 * nRfr, Re.im + e1 * Rf.im + e2 * nRfi};
        Lf = Lf2; Uf = Uf2; Df = Df2; Rf = Rf2;
        Le = Le2; Ue = Ue2; De = De2; Re = Re2;
    }
    // strides 2, 4, .., 2 LPL / 2: unknowns of the same kind, lanes r -/+ q
#pragma unroll
    for (int q = 1; q < LPL; q <<= 1) {
        const int rm = (r - q) & (LPL - 1), rp = (r + q) & (LPL - 1);
        T *Ls[2] = {&Lf, &Le}, *Ds[2] = {&Df, &De}, *Us[2] = {&Uf, &Ue};
        cplx<T> *Rs[2] = {&Rf, &Re};
#pragma unroll
        for (int kind = 0; kind < 2; ++kind) {
            T &L = *Ls[kind], &D = *Ds[kind], &U = *Us[kind];
            cplx<T> &R = *Rs[kind];
            const T mL = __shfl_sync(0xffffffffu, L, rm, LPL);
            const T mD = __shfl_sync(0xffffffffu, D, rm, LPL);
            const T mU = __shfl_sync(0xffffffffu, U, rm, LPL);
            const T mRr = __shfl_sync(0xffffffffu, R.re, rm, LPL);
            const T mRi = __shfl_sync(0xffffffffu, R.im, rm, LPL);
            const T pL = __shfl_sync(0xffffffffu, L, rp, LPL);
            const T pD = __shfl_sync(0xffffffffu, D, rp, LPL);
            const T pU = __shfl_sync(0xffffffffu, U, rp, LPL);
            const T pRr = __shfl_sync(0xffffffffu, R.re, rp, LPL);
            const T pRi = __shfl_sync(0xffffffffu, R.im, rp, LPL);
            const T k1 = -L * rcp(mD), k2 = -U * rcp(pD);
            const T D2 = D + k1 * mU + k2 * pL;
            R = cplx<T>{R.re + k1 * mRr + k2 * pRr, R.im + k1 * mRi + k2 * pRi};
            L = k1 * mL;
            U = k2 * pU;
            D = D2;
        }
    }
    // every equation now couples only to itself (cyclic) or to nothing
    const T fi = rcp(Df + Lf + Uf), ei = rcp(De + Le + Ue);
    const cplx<T> xF{Rf.re * fi, Rf.im * fi}, xE{Re.re * ei, Re.im * ei};
    d[0] = xF;
    d[E - 1] = xE;
    {
        cplx<T> x = xE;
#pragma unroll
        for (int i = E - 2; i >= 1; --i) {
            x = cplx<T>{d[i].re - at[i] * xF.re - ct[i] * x.re,
                        d[i].im - at[i] * xF.im - ct[i] * x.im};
            d[i] = x;
        }
    }
#pragma unroll
    for (int i = 0; i < E; ++i) S[pos(s0 + i, w)] = d[i];
    __syncthreads();
    const unsigned char *ex = exact + (size_t)ky * sk + x0;
    for (int e = t; e < nz * NL; e += 256) {
        const int z = e / NL, w2 = e - z * NL;
        if (!ex[w2]) col[(size_t)z * plane + w2] = scale * S[pos(z, w2)];
    }
}

size_t smem_exact(int nz, int P) {
    const size_t rs = 2 * P + 1;
    return sizeof(cplx<double>) * (nz + rs) + sizeof(double) * (2 * (size_t)nz + 3 * rs);
}

// about sqrt(nz) chunks: the chunk sweeps and the serial reduced system
// (FP64 divisions on its critical path) then have similar lengths
int exact_chunks(int nz) {
    int P = 16;
    if (P > (nz - 1) / 3) P = (nz - 1) / 3;
    return P < 1 ? 1 : P;
}

// Complex-to-real inverse DFT along x of RY spectrum rows into dst: the
// rows (kx <= mx) are copied asynchronously, recombined into the half-length
// complex sequence Z_kx = (X_kx + conj X_{mx-kx}) + i conj(w^kx) (X_kx -
// conj X_{mx-kx}), inverse transformed, and the complex result stored as the
// interleaved real row.
template <typename T, int RY>
FSEI_D void
k_irfft_x(GridDev g, const cplx<T> *__restrict__ spec, T *__restrict__ dst,
          const cplx<T> *__restrict__ twx, const cplx<T> *__restrict__ twpost, FftPlanDev fp) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nx = g.nx, ny = g.ny, mx = g.mx, sk = g.sk;
    const int ls = fft_x_ls(mx);
    const int ss = irfft_stage_row(mx);
    const int bls = fft_x_bls(mx);
    cplx<T> *A = reinterpret_cast<cplx<T> *>(smraw);
    cplx<T> *B = A + (size_t)RY * ls;
    cplx<T> *TW = B + (size_t)RY * bls;
    cplx<T> *TP = TW + fft_x_ls(mx);
    cplx<T> *S = TP + fft_x_ls(mx + 1);
    const int nby = ny / RY;
    const int k = blockIdx.x / nby, j0 = (blockIdx.x % nby) * RY;
    copy_rows_async(S, ss * sizeof(cplx<T>), spec + ((size_t)k * ny + j0) * sk,
                    (size_t)sk * sizeof(cplx<T>), RY, ss * (int)sizeof(cplx<T>));
    stage_x_twiddles(TW, TP, twx, twpost, mx);
    cp_async_wait_all();
    __syncthreads();
    for (int e = threadIdx.x; e < RY * mx; e += blockDim.x) {
        const int r = ddiv(e, mx), kx = e - r * mx;
        const cplx<T> *row = S + (size_t)r * ss;
        const cplx<T> xk = row[kx];
        const cplx<T> xm = conj(row[mx - kx]);
        const cplx<T> ev = xk + xm;
        const cplx<T> od = (xk - xm) * conj(TP[kx]);
        A[r * ls + kx] = ev + mul_i<T, 1>(od);
    }
    __syncthreads();
    const cplx<T> *R = fft_lines_fast<T, 1, false>(A, B, 1, ls, bls, RY, fp, TW);
    const bool v16 = ((nx * sizeof(T)) & 15) == 0;
    for (int r = 0; r < RY; ++r) {
        T *drow = dst + ((size_t)k * ny + j0 + r) * nx;
        const T *srow = reinterpret_cast<const T *>(R + (size_t)r * ls);
        if (v16) {
            const int per = nx * (int)sizeof(T) / 16;
            for (int c = threadIdx.x; c < per; c += blockDim.x)
                reinterpret_cast<uint4 *>(drow)[c] = reinterpret_cast<const uint4 *>(srow)[c];
        } else {
            for (int i = threadIdx.x; i < nx; i += blockDim.x) drow[i] = srow[i];
        }
    }
}

// The inverse x transform for power-of-two mx = N1 N2 <= 256 without
// staging tiles: pass 1 (item: row r, n2) loads the spectrum values X_m and
// X_{mx-m} of its N1 indices m = N1' N2 + n2 straight from global memory,
// forms the half-length sequence Z_m = (X_m + conj X_{mx-m}) + i conj(w^m)
// (X_m - conj X_{mx-m}) in registers (as k_irfft_x does), applies the
// in-register DFT and the twiddles and writes the transposed values to
// shared memory; pass 2 (item: r, k1) applies the second DFT and stores z_m
// as the real pair (x_2m, x_2m+1) straight to the output row.
// Single precision: 3 blocks per SM (80 registers, no spills; 256^3: 45 ->
// 39 us against 92 registers and 2 blocks).
template <typename T, int RY, int N1, int N2>
FSEI_D void
k_irfft_x_2p(GridDev g, const cplx<T> *__restrict__ spec, T *__restrict__ dst,
             const cplx<T> *__restrict__ twx, const cplx<T> *__restrict__ twpost) {
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_wait();
    pdl_trigger();
    constexpr int MX = N1 * N2;
    constexpr int BL = N2 * (N1 + 1);
    const int nx = g.nx, ny = g.ny, sk = g.sk;
    cplx<T> *B = reinterpret_cast<cplx<T> *>(smraw);   // RY rows of BL
    cplx<T> *TW = B + (size_t)RY * BL;                 // w^m, m < MX
    cplx<T> *TP = TW + MX;                             // w_nx^m, m <= MX
    const int nby = ny / RY;
    const int k = blockIdx.x / nby, j0 = (blockIdx.x % nby) * RY;
    const cplx<T> *src = spec + ((size_t)k * ny + j0) * sk;
    const int t = threadIdx.x;
    const bool on1 = t < RY * N2;
    const int r1 = t / N2, n2 = t - r1 * N2;
    cplx<T> xa[N1], xb[N1];
    if (on1) {
        const cplx<T> *row = src + (size_t)r1 * sk;
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            const int m = a * N2 + n2;
            xa[a] = row[m];
            xb[a] = row[MX - m];
        }
    }
    for (int m = t; m < MX; m += blockDim.x) TW[m] = twx[m];
    for (int m = t; m <= MX; m += blockDim.x) TP[m] = twpost[m];
    __syncthreads();
    if (on1) {
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            const int m = a * N2 + n2;
            const cplx<T> xk = xa[a], xm = conj(xb[a]);
            const cplx<T> ev = xk + xm;
            const cplx<T> od = (xk - xm) * conj(TP[m]);
            xa[a] = ev + mul_i<T, 1>(od);
        }
        dft_reg<T, N1, 1>(xa, TW, MX);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) xa[k1] = xa[k1] * conj(TW[n2 * k1]);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) B[r1 * BL + n2 * (N1 + 1) + k1] = xa[k1];
    }
    __syncthreads();
    if (t < RY * N1) {
        const int r2 = t / N1, k1 = t - r2 * N1;
        cplx<T> y[N2];
#pragma unroll
        for (int q = 0; q < N2; ++q) y[q] = B[r2 * BL + q * (N1 + 1) + k1];
        dft_reg<T, N2, 1>(y, TW, MX);
        cplxa<T> *drow = reinterpret_cast<cplxa<T> *>(dst + ((size_t)k * ny + j0 + r2) * nx);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            cplxa<T> v;
            v.re = y[k2].re;
            v.im = y[k2].im;
            drow[k1 + N1 * k2] = v;
        }
    }
}

}  // namespace

// the kernels with their launch bounds
template <typename T, int MODE, int RY>
constexpr Kernel<k_rfft_x<T, MODE, RY>, 256, (sizeof(T) == 4 ? 4 : 1)> K_rfft_x{};
template <typename T, int SIGN> constexpr Kernel<k_fft_y<T, SIGN>, 256, 0> K_fft_y{};
// single precision, first-pass DFTs of up to 16 points: 4 blocks per SM (64
// registers, as without the second turn of pairs the wider tiles need)
template <typename T, int SIGN, int N1, int N2>
constexpr Kernel<k_fft_y_2p<T, SIGN, N1, N2>, 256, (sizeof(T) == 4 && N1 <= 16 ? 4 : 0)>
    K_fft_y_2p{};
template <typename T> constexpr Kernel<k_poisson_z<T>, 512, 0> K_poisson_z{};
template <typename T> constexpr Kernel<k_poisson_exact<T>, 64, 0> K_poisson_exact{};
template <typename T> constexpr Kernel<k_poisson_exact_f<T>, 32, 0> K_poisson_exact_f{};
// single precision: 3 blocks per SM for chunks of up to 16 rows; longer
// chunks (24 rows of the 768-row lines) need the registers of 2 blocks
template <typename T, int E, int LPL>
constexpr Kernel<k_poisson_zl<T, E, LPL>, 256, (sizeof(T) == 4 && E <= 16 ? 3 : 2)>
    K_poisson_zl{};
template <typename T, int RY> constexpr Kernel<k_irfft_x<T, RY>, 256, 0> K_irfft_x{};
template <typename T, int RY, int N1, int N2>
constexpr Kernel<k_irfft_x_2p<T, RY, N1, N2>, 256, (sizeof(T) == 4 ? 3 : 1)> K_irfft_x_2p{};

// x transforms: two line buffers, the twiddle tables and (inverse only) the
// staged spectrum rows; ry rows per block
template <typename T> size_t smem_rfft_x(const GridDev &g, int ry) {
    return sizeof(cplx<T>) * ((size_t)ry * (fft_x_ls(g.mx) + fft_x_bls(g.mx)) + fft_x_ls(g.mx) +
                              fft_x_ls(g.mx + 1));
}
template <typename T> size_t smem_irfft_x(const GridDev &g, int ry) {
    return smem_rfft_x<T>(g, ry) + sizeof(cplx<T>) * (size_t)ry * irfft_stage_row(g.mx);
}
template <typename T> size_t smem_fft_x(const GridDev &g, const Work<T> &W) {
    return smem_irfft_x<T>(g, W.ry_fft);
}
template <typename T> size_t smem_fft_y(const GridDev &g, const Work<T> &W) {
    return sizeof(cplx<T>) * (2 * (size_t)W.tkx * g.ny + g.ny);
}
template <typename T> size_t smem_poisson(const GridDev &g, const Work<T> &W) {
    const size_t rs = 2 * W.pz_poisson + 1;
    return sizeof(cplx<T>) * ((size_t)g.nz * W.tkx + W.tkx * rs) +
           sizeof(T) * (2 * (size_t)g.nz * W.tkx + 3 * W.tkx * rs + W.tkx + 3 * (size_t)g.nz);
}

// Launch geometry of the transforms and the z solve: rows per block of the x
// transforms (up to 8 in single, 4 in double precision, dividing ny) and kx
// columns per block of the y transform and z solve (up to 128 bytes of
// complex values per row), each the largest whose shared memory, computed
// exactly, fits the device limit.
int zl_candidates(const GridDev &g, int elem_size, int (*out)[2], int cap) {
    // instantiated splits with nz = LPL E, 16 lanes per line first (fewer
    // reduction levels; at 256^3 measured 41 against 59 us for 32 lanes of
    // half the rows); in double at most 8 rows per lane (registers)
    static const int cand[][2] = {{16, 4}, {16, 6}, {16, 8}, {16, 12}, {16, 16},
                                  {16, 24}, {32, 8}, {32, 16}, {32, 24}};
    int n = 0;
    for (const auto &c : cand) {
        if (elem_size == 8 && c[1] > 8) continue;
        if (g.nz == c[0] * c[1] && g.sk % (256 / c[0]) == 0 && n < cap) {
            out[n][0] = c[0];
            out[n][1] = c[1];
            ++n;
        }
    }
    return n;
}

template <typename T> void poisson_geometry(const GridDev &g, Work<T> &W) {
    const size_t lim = (size_t)smem_optin() - 2048;
    const int tsz = (int)sizeof(T);
    W.ry_fft = 1;
    for (int r = tsz == 8 ? 4 : 16; r >= 1; r /= 2)
        if (g.ny % r == 0) { W.ry_fft = r; break; }
    while (W.ry_fft > 1 && smem_fft_x<T>(g, W) > lim) W.ry_fft /= 2;
    // lane-resident z solve: the first applicable (lanes per line, rows per
    // lane) split; the grid's autotuner may pick another
    W.zl_lpl = W.zl_e = 0;
    {
        int c[4][2];
        if (zl_candidates(g, tsz, c, 4) > 0) {
            W.zl_lpl = c[0][0];
            W.zl_e = c[0][1];
        }
    }
    W.tkx = 128 / (2 * tsz);
    for (;;) {
        W.pz_poisson = 256 / W.tkx;
        if (W.pz_poisson > g.nz / 3) W.pz_poisson = g.nz / 3;
        if (W.pz_poisson < 1) W.pz_poisson = 1;
        if (W.tkx <= 2 || (smem_poisson<T>(g, W) <= lim && smem_fft_y<T>(g, W) <= lim)) break;
        W.tkx /= 2;
    }
    W.ry_rfft = W.ry_fft;
    W.tkx_fft = W.tkx;
    {
        const int n1 = fft_split_n1(g.ny);
        while (n1 && W.tkx_fft > 1 && W.tkx_fft * n1 > 256) W.tkx_fft /= 2;
    }
}

template <typename T, int MODE, int RY>
void rfft_x_ry(const GridDev &g, Work<T> &W, const StepScalars *sc, const T *src, cudaStream_t st) {
    const int blocks = g.nz * (g.ny / RY);
    K_rfft_x<T, MODE, RY>.launch(W.pdl != 0, dim3(blocks), dim3(256), smem_rfft_x<T>(g, RY), st,
                                 g, W.q0, W.q1, W.q2, src, W.spec, W.twx, W.twpost, W.fpx, sc);
}

template <typename T, int MODE>
void rfft_x_mode(const GridDev &g, Work<T> &W, const StepScalars *sc, const T *src,
                 cudaStream_t st) {
    switch (W.ry_rfft) {
    case 16: rfft_x_ry<T, MODE, 16>(g, W, sc, src, st); break;
    case 8: rfft_x_ry<T, MODE, 8>(g, W, sc, src, st); break;
    case 4: rfft_x_ry<T, MODE, 4>(g, W, sc, src, st); break;
    case 2: rfft_x_ry<T, MODE, 2>(g, W, sc, src, st); break;
    default: rfft_x_ry<T, MODE, 1>(g, W, sc, src, st); break;
    }
}

template <typename T> void launch_rfft_x(const GridDev &g, Work<T> &W, const StepScalars *sc,
                                         const T *src, int mode, cudaStream_t st) {
    if (mode == 0) rfft_x_mode<T, 0>(g, W, sc, nullptr, st);
    else rfft_x_mode<T, 1>(g, W, sc, src, st);
}

template <typename T, int SIGN>
bool fft_y_2p_launch(const GridDev &g, Work<T> &W, cudaStream_t st) {
    const int tk = W.tkx_fft;
    const int n1 = fft_split_n1(g.ny);
    if (!n1 || tk < 1 || g.sk % tk || tk * n1 > 512 || tk * (g.ny / n1) > 512) return false;
    const int blocks = g.nz * (g.sk / tk);
    const size_t sm = sizeof(cplx<T>) * ((size_t)g.ny * tk + g.ny);
    // at most 256 threads: wider tiles take their pairs in two turns
    const int thr = tk * n1 < 256 ? tk * n1 : 256;
    const bool pdl = W.pdl != 0;
    switch (g.ny) {
#define FSEI_FY(N1_, N2_)                                                                      \
    K_fft_y_2p<T, SIGN, N1_, N2_>.launch(pdl, dim3(blocks), dim3(thr), sm, st, g, W.spec, W.twy, tk)
    case 16: FSEI_FY(4, 4); return true;
    case 32: FSEI_FY(8, 4); return true;
    case 64: FSEI_FY(8, 8); return true;
    case 128: FSEI_FY(16, 8); return true;
    case 256: FSEI_FY(16, 16); return true;
    case 512: FSEI_FY(32, 16); return true;
    case 12: FSEI_FY(4, 3); return true;
    case 24: FSEI_FY(6, 4); return true;
    case 48: FSEI_FY(8, 6); return true;
    case 96: FSEI_FY(12, 8); return true;
    case 192: FSEI_FY(16, 12); return true;
    case 384: FSEI_FY(24, 16); return true;
#undef FSEI_FY
    default: return false;
    }
}

template <typename T> void launch_fft_y(const GridDev &g, Work<T> &W, int inverse, cudaStream_t st) {
    if (inverse ? fft_y_2p_launch<T, 1>(g, W, st) : fft_y_2p_launch<T, -1>(g, W, st)) return;
    const int blocks = g.nz * (g.sk / W.tkx);
    if (inverse)
        K_fft_y<T, 1>.launch(false, dim3(blocks), dim3(256), smem_fft_y(g, W), st, g, W.spec, W.twy,
                             W.fpy, W.tkx);
    else
        K_fft_y<T, -1>.launch(false, dim3(blocks), dim3(256), smem_fft_y(g, W), st, g, W.spec,
                              W.twy, W.fpy, W.tkx);
}

template <typename T> void launch_poisson_z(const GridDev &g, Work<T> &W, cudaStream_t st,
                                            int compat) {
    const int blocks = g.ny * (g.sk / W.tkx);
    const int threads = ((W.tkx * W.pz_poisson + 31) / 32) * 32;
    const double scale = 1.0 / ((double)g.nx * g.ny);
    if (W.xa && W.zl_lpl) {
        // one launch: the exactly solved modes in its first blocks
        const int nl = 256 / W.zl_lpl;
        const size_t sm1 = sizeof(cplx<T>) * (size_t)g.nz * nl +
                           sizeof(ZCoef<T>) * (size_t)(g.nz + g.nz / W.zl_e);
        const size_t sm2 = sizeof(cplx<double>) * (size_t)g.nz;
        const size_t sm = sm1 > sm2 ? sm1 : sm2;
        const int grid = W.n_nzm + g.ny * (g.sk / nl);
        const T tsc = T(scale);
#define FSEI_ZL(E_, L_)                                                                        \
    if (W.zl_e == E_ && W.zl_lpl == L_) {                                                      \
        K_poisson_zl<T, E_, L_>.launch(W.pdl != 0, dim3(grid), dim3(256), sm, st, g, W.spec,     \
                                       W.lamx, W.lamy, W.exact, tsc, W.n_nzm, W.nzm, W.xa,    \
                                       W.xm, W.xc, W.xz, W.xs, scale, compat, W.zlen);        \
        return;                                                                                \
    }
        FSEI_ZL(4, 16) FSEI_ZL(6, 16) FSEI_ZL(8, 16) FSEI_ZL(8, 32)
        if constexpr (sizeof(T) == 4) {
            FSEI_ZL(12, 16) FSEI_ZL(16, 16) FSEI_ZL(24, 16) FSEI_ZL(16, 32) FSEI_ZL(24, 32)
        }
#undef FSEI_ZL
    }
    // exact modes first: they read the untouched right-hand side, and
    // k_poisson_z leaves them alone
    if (W.xa) {
        K_poisson_exact_f<T>.launch(false, dim3(W.n_nzm), dim3(32), sizeof(cplx<double>) * g.nz,
                                    st, g, W.spec, W.nzm, W.xa, W.xm, W.xc, W.xz, W.xs, scale,
                                    compat, W.zlen);
    } else {
        const int Pe = exact_chunks(g.nz);
        K_poisson_exact<T>.launch(false, dim3(W.n_nzm), dim3(64), smem_exact(g.nz, Pe), st, g,
                                  W.spec, W.nzm, W.lamx_d, W.lamy_d, scale, compat, Pe);
    }
    K_poisson_z<T>.launch(false, dim3(blocks), dim3(threads), smem_poisson(g, W), st, g, W.spec,
                          W.lamx, W.lamy, W.exact, W.tkx, W.pz_poisson, T(scale));
}

template <typename T, int RY>
void irfft_x_ry(const GridDev &g, Work<T> &W, T *dst, cudaStream_t st) {
    const int blocks = g.nz * (g.ny / RY);
    K_irfft_x<T, RY>.launch(false, dim3(blocks), dim3(256), smem_irfft_x<T>(g, RY), st, g, W.spec,
                            dst, W.twx, W.twpost, W.fpx);
}

template <typename T, int RY>
bool irfft_x_2p_launch(const GridDev &g, Work<T> &W, T *dst, cudaStream_t st) {
    const int n1 = fft_split_n1(g.mx);
    if (!n1 || W.ry_fft != RY || RY * n1 > 256) return false;
    const int blocks = g.nz * (g.ny / RY);
    const size_t sm = sizeof(cplx<T>) * ((size_t)RY * (g.mx / n1) * (n1 + 1) + 2 * g.mx + 1);
    const int thr = RY * n1;
    const bool pdl = W.pdl != 0;
    switch (g.mx) {
#define FSEI_IX(N1_, N2_)                                                                      \
    K_irfft_x_2p<T, RY, N1_, N2_>.launch(pdl, dim3(blocks), dim3(thr), sm, st, g, W.spec, dst,   \
                                         W.twx, W.twpost)
    case 16: FSEI_IX(4, 4); return true;
    case 32: FSEI_IX(8, 4); return true;
    case 64: FSEI_IX(8, 8); return true;
    case 128: FSEI_IX(16, 8); return true;
    case 256: FSEI_IX(16, 16); return true;
    case 12: FSEI_IX(4, 3); return true;
    case 24: FSEI_IX(6, 4); return true;
    case 48: FSEI_IX(8, 6); return true;
    case 96: FSEI_IX(12, 8); return true;
    case 192: FSEI_IX(16, 12); return true;
#undef FSEI_IX
    default: return false;
    }
}

template <typename T> void launch_irfft_x(const GridDev &g, Work<T> &W, T *dst, cudaStream_t st) {
    if (irfft_x_2p_launch<T, sizeof(T) == 4 ? 16 : 4>(g, W, dst, st)) return;
    switch (W.ry_fft) {
    case 16: irfft_x_ry<T, 16>(g, W, dst, st); break;
    case 8: irfft_x_ry<T, 8>(g, W, dst, st); break;
    case 4: irfft_x_ry<T, 4>(g, W, dst, st); break;
    case 2: irfft_x_ry<T, 2>(g, W, dst, st); break;
    default: irfft_x_ry<T, 1>(g, W, dst, st); break;
    }
}

template <typename T> void set_smem_limits_poisson(const GridDev &g, const Work<T> &W) {
    (void)0;  // every kernel of this file gets an attribute below, which loads it
    raise_smem_limit(K_rfft_x<T, 0, 1>.solo());
    raise_smem_limit(K_rfft_x<T, 0, 2>.solo());
    raise_smem_limit(K_rfft_x<T, 0, 4>.solo());
    raise_smem_limit(K_rfft_x<T, 0, 8>.solo());
    raise_smem_limit(K_rfft_x<T, 0, 16>.solo());
    raise_smem_limit(K_rfft_x<T, 1, 16>.solo());
    raise_smem_limit(K_irfft_x<T, 16>.solo());
    {
        constexpr int R = sizeof(T) == 4 ? 16 : 4;
        raise_smem_limit(K_irfft_x_2p<T, R, 4, 4>.solo());
        raise_smem_limit(K_irfft_x_2p<T, R, 8, 4>.solo());
        raise_smem_limit(K_irfft_x_2p<T, R, 8, 8>.solo());
        raise_smem_limit(K_irfft_x_2p<T, R, 16, 8>.solo());
        raise_smem_limit(K_irfft_x_2p<T, R, 16, 16>.solo());
        raise_smem_limit(K_irfft_x_2p<T, R, 4, 3>.solo());
        raise_smem_limit(K_irfft_x_2p<T, R, 6, 4>.solo());
        raise_smem_limit(K_irfft_x_2p<T, R, 8, 6>.solo());
        raise_smem_limit(K_irfft_x_2p<T, R, 12, 8>.solo());
        raise_smem_limit(K_irfft_x_2p<T, R, 16, 12>.solo());
    }
    raise_smem_limit(K_rfft_x<T, 1, 1>.solo());
    raise_smem_limit(K_rfft_x<T, 1, 2>.solo());
    raise_smem_limit(K_rfft_x<T, 1, 4>.solo());
    raise_smem_limit(K_rfft_x<T, 1, 8>.solo());
    raise_smem_limit(K_irfft_x<T, 1>.solo());
    raise_smem_limit(K_irfft_x<T, 2>.solo());
    raise_smem_limit(K_irfft_x<T, 4>.solo());
    raise_smem_limit(K_irfft_x<T, 8>.solo());
    raise_smem_limit(K_fft_y<T, 1>.solo());
    raise_smem_limit(K_fft_y<T, -1>.solo());
    raise_smem_limit(K_fft_y_2p<T, 1, 4, 4>.solo());
    raise_smem_limit(K_fft_y_2p<T, -1, 4, 4>.solo());
    raise_smem_limit(K_fft_y_2p<T, 1, 8, 4>.solo());
    raise_smem_limit(K_fft_y_2p<T, -1, 8, 4>.solo());
    raise_smem_limit(K_fft_y_2p<T, 1, 8, 8>.solo());
    raise_smem_limit(K_fft_y_2p<T, -1, 8, 8>.solo());
    raise_smem_limit(K_fft_y_2p<T, 1, 16, 8>.solo());
    raise_smem_limit(K_fft_y_2p<T, -1, 16, 8>.solo());
    raise_smem_limit(K_fft_y_2p<T, 1, 16, 16>.solo());
    raise_smem_limit(K_fft_y_2p<T, -1, 16, 16>.solo());
    raise_smem_limit(K_fft_y_2p<T, 1, 32, 16>.solo());
    raise_smem_limit(K_fft_y_2p<T, -1, 32, 16>.solo());
    raise_smem_limit(K_fft_y_2p<T, 1, 4, 3>.solo());
    raise_smem_limit(K_fft_y_2p<T, -1, 4, 3>.solo());
    raise_smem_limit(K_fft_y_2p<T, 1, 6, 4>.solo());
    raise_smem_limit(K_fft_y_2p<T, -1, 6, 4>.solo());
    raise_smem_limit(K_fft_y_2p<T, 1, 8, 6>.solo());
    raise_smem_limit(K_fft_y_2p<T, -1, 8, 6>.solo());
    raise_smem_limit(K_fft_y_2p<T, 1, 12, 8>.solo());
    raise_smem_limit(K_fft_y_2p<T, -1, 12, 8>.solo());
    raise_smem_limit(K_fft_y_2p<T, 1, 16, 12>.solo());
    raise_smem_limit(K_fft_y_2p<T, -1, 16, 12>.solo());
    raise_smem_limit(K_fft_y_2p<T, 1, 24, 16>.solo());
    raise_smem_limit(K_fft_y_2p<T, -1, 24, 16>.solo());
    raise_smem_limit(K_poisson_z<T>.solo());
    raise_smem_limit(K_poisson_exact<T>.solo());
    raise_smem_limit(K_poisson_exact_f<T>.solo());
    raise_smem_limit(K_poisson_zl<T, 4, 16>.solo());
    raise_smem_limit(K_poisson_zl<T, 6, 16>.solo());
    raise_smem_limit(K_poisson_zl<T, 8, 16>.solo());
    raise_smem_limit(K_poisson_zl<T, 8, 32>.solo());
    if constexpr (sizeof(T) == 4) {
        raise_smem_limit(K_poisson_zl<T, 12, 16>.solo());
        raise_smem_limit(K_poisson_zl<T, 16, 16>.solo());
        raise_smem_limit(K_poisson_zl<T, 24, 16>.solo());
        raise_smem_limit(K_poisson_zl<T, 16, 32>.solo());
        raise_smem_limit(K_poisson_zl<T, 24, 32>.solo());
    }
}

template <typename T> int schedule_candidates(const GridDev &g, int knob, int (*out)[2], int cap) {
    const size_t lim = (size_t)smem_optin() - 2048;
    const int tsz = (int)sizeof(T);
    int n = 0;
    auto put = [&](int a, int b) {
        if (n < cap) {
            out[n][0] = a;
            out[n][1] = b;
            ++n;
        }
    };
    switch (knob) {
    case SK_RHS: {
        // (cells per lane, rows per strip): the default (8 cells per lane in
        // single precision on rows wider than 256 cells, 4 otherwise; one
        // row per lane) first, then the strips of the marched kernel
        int c[5];
        const int m = rhs_cpl_candidates(g, tsz, c, 5);
        const int def = (tsz == 4 && g.nx > 256) ? 8 : 4;
        int order[5], no = 0;
        for (int i = 0; i < m; ++i)
            if (c[i] == def) order[no++] = c[i];
        for (int i = 0; i < m; ++i)
            if (c[i] != def) order[no++] = c[i];
        for (int i = 0; i < no; ++i) put(order[i], 0);
        const int strips[3] = {8, 4, 16};
        for (int i = 0; i < no; ++i)
            for (int S : strips)
                if (rhs_strip_admissible(g, tsz, order[i], S)) put(order[i], S);
        break;
    }
    case SK_ZL: {
        int c[9][2];
        const int m = zl_candidates(g, tsz, c, 9);
        for (int i = 0; i < m; ++i) put(c[i][0], c[i][1]);
        break;
    }
    case SK_RFFT: {
        // rows per block: powers of two dividing ny whose buffers fit; the
        // default (the largest up to 16 in single, 4 in double precision)
        // first
        Work<T> W;
        memset(&W, 0, sizeof W);
        poisson_geometry<T>(g, W);
        put(W.ry_rfft, 0);
        for (int r = 16; r >= 2; r /= 2)
            if (r != W.ry_rfft && g.ny % r == 0 && smem_rfft_x<T>(g, r) <= lim) put(r, 0);
        break;
    }
    case SK_FFTY: {
        // kx columns per block of the two-pass y transform: tkx N1 pairs of
        // the second pass, 32 to 512 (at most 256 threads, two turns above)
        const int n1 = fft_split_n1(g.ny);
        if (!n1) break;
        Work<T> W;
        memset(&W, 0, sizeof W);
        poisson_geometry<T>(g, W);
        put(W.tkx_fft, 0);
        for (int t = 32; t >= 2; t /= 2)
            if (t != W.tkx_fft && g.sk % t == 0 && t * n1 <= 512 && t * (g.ny / n1) <= 512 &&
                t * n1 >= 32 &&
                sizeof(cplx<T>) * ((size_t)g.ny * t + g.ny) <= lim)
                put(t, 0);
        break;
    }
    case SK_ZSW: {
        // x columns per lane of the z sweep: 1 first, 2 for chunks of up to
        // 16 rows
        int chunk, P, tx;
        sweep_geometry(g.nz, chunk, P, tx);
        if (chunk <= 16) {
            put(1, 0);
            put(2, 0);
        }
        break;
    }
    case SK_PROJ: {
        // row passes per thread of the 16-byte vector projection
        if (g.nx % (16 / tsz)) break;
        const int opts[4] = {4, 2, 8, 1};
        for (int m : opts) put(m, 0);
        break;
    }
    default: break;
    }
    return n;
}

template <typename T> Schedule schedule_of(const GridDev &g, const Work<T> &W) {
    Schedule s;
    memset(&s, 0, sizeof s);
    int c[1][2];
    if (schedule_candidates<T>(g, SK_RHS, c, 1)) {
        s.rhs_cpl = W.rhs_cpl ? W.rhs_cpl : c[0][0];
        s.rhs_strip = W.rhs_strip;
    }
    s.zl_lpl = W.zl_lpl;
    s.zl_e = W.zl_e;
    s.ry_rfft = W.ry_rfft;
    if (schedule_candidates<T>(g, SK_FFTY, c, 1)) s.tkx_fft = W.tkx_fft;
    if (schedule_candidates<T>(g, SK_PROJ, c, 1)) s.proj_mult = W.proj_mult ? W.proj_mult : 4;
    if (schedule_candidates<T>(g, SK_ZSW, c, 1)) s.zsw_cols = W.zsw_cols ? W.zsw_cols : 1;
    return s;
}

template <typename T> void apply_schedule(Work<T> &W, const Schedule &s) {
    W.rhs_cpl = s.rhs_cpl;
    W.rhs_strip = s.rhs_strip;
    W.zl_lpl = s.zl_lpl;
    W.zl_e = s.zl_e;
    if (s.ry_rfft) W.ry_rfft = s.ry_rfft;
    if (s.tkx_fft) W.tkx_fft = s.tkx_fft;
    W.proj_mult = s.proj_mult;
    W.zsw_cols = s.zsw_cols;
}

#define FSEI_INST(T)                                                                           \
    template size_t smem_fft_x<T>(const GridDev &, const Work<T> &);                          \
    template size_t smem_fft_y<T>(const GridDev &, const Work<T> &);                          \
    template size_t smem_poisson<T>(const GridDev &, const Work<T> &);                        \
    template void poisson_geometry<T>(const GridDev &, Work<T> &);                             \
    template int schedule_candidates<T>(const GridDev &, int, int (*)[2], int);                 \
    template Schedule schedule_of<T>(const GridDev &, const Work<T> &);                        \
    template void apply_schedule<T>(Work<T> &, const Schedule &);                              \
    template void launch_rfft_x<T>(const GridDev &, Work<T> &, const StepScalars *, const T *, \
                                   int, cudaStream_t);                                        \
    template void launch_fft_y<T>(const GridDev &, Work<T> &, int, cudaStream_t);              \
    template void launch_poisson_z<T>(const GridDev &, Work<T> &, cudaStream_t, int);          \
    template void launch_irfft_x<T>(const GridDev &, Work<T> &, T *, cudaStream_t);            \
    template void set_smem_limits_poisson<T>(const GridDev &, const Work<T> &);
FSEI_INST(float)
FSEI_INST(double)
#undef FSEI_INST

}  // namespace fsei
