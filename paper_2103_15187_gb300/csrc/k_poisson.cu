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
#include "kernels.cuh"
#include "tri.cuh"

namespace fsei {

namespace {

FSEI_D size_t fid(int i, int j, int k, int nx, int ny) {
    return ((size_t)k * ny + j) * nx + i;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(512)
k_rfft_x(GridDev g, const T *__restrict__ q0, const T *__restrict__ q1,
         const T *__restrict__ q2, const T *__restrict__ src, cplx<T> *__restrict__ spec,
         const cplx<T> *__restrict__ twx, const cplx<T> *__restrict__ twpost, FftPlanDev fp,
         const StepScalars *sc, int ry) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nx = g.nx, ny = g.ny, nz = g.nz, mx = g.mx, sk = g.sk;
    const int ls = mx | 1;
    cplx<T> *A = reinterpret_cast<cplx<T> *>(smraw);
    cplx<T> *B = A + (size_t)ry * ls;
    const int nby = ny / ry;
    const int k = blockIdx.x / nby, j0 = (blockIdx.x % nby) * ry;
    T invdt = T(1);
    if (MODE == 0) invdt = T(1.0 / sc->dt);
    const bool hasup = !g.walls || k < nz - 1;
    const int ku = k == nz - 1 ? 0 : k + 1;
    const T idx = T(g.idx), idy = T(g.idy);
    const T idzk = Metric<T>::idz(g)[k];
    for (int e = threadIdx.x; e < ry * nx; e += blockDim.x) {
        const int r = e / nx, i = e - r * nx, j = j0 + r;
        const size_t c = fid(i, j, k, nx, ny);
        T s;
        if (MODE == 0) {
            const int ip = i == nx - 1 ? 0 : i + 1, jp = j == ny - 1 ? 0 : j + 1;
            const T wku = hasup ? q2[fid(i, j, ku, nx, ny)] : T(0);
            s = ((q0[fid(ip, j, k, nx, ny)] - q0[c]) * idx + (q1[fid(i, jp, k, nx, ny)] - q1[c]) * idy +
                 (wku - q2[c]) * idzk) * invdt;
        } else {
            s = src[c];
        }
        reinterpret_cast<T *>(A + (size_t)r * ls)[i] = s;
    }
    __syncthreads();
    const cplx<T> *R = fft_lines<T, -1>(A, B, 1, ls, ry, fp, twx, false);
    const T hf = T(0.5);
    for (int e = threadIdx.x; e < ry * (mx + 1); e += blockDim.x) {
        const int r = e / (mx + 1), kx = e - r * (mx + 1);
        const cplx<T> zk = R[r * ls + (kx == mx ? 0 : kx)];
        const cplx<T> zc = conj(R[r * ls + (kx == 0 ? 0 : mx - kx)]);
        const cplx<T> ev = hf * (zk + zc);
        const cplx<T> od = mul_i<T, -1>(hf * (twpost[kx] * (zk - zc)));
        spec[((size_t)k * ny + j0 + r) * sk + kx] = ev + od;
    }
}

template <typename T, int SIGN>
__global__ void __launch_bounds__(512)
k_fft_y(GridDev g, cplx<T> *__restrict__ spec, const cplx<T> *__restrict__ twy, FftPlanDev fp,
        int tkx) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int ny = g.ny, sk = g.sk;
    cplx<T> *A = reinterpret_cast<cplx<T> *>(smraw);
    cplx<T> *B = A + (size_t)ny * tkx;
    const int nkt = sk / tkx;
    const int k = blockIdx.x / nkt, x0 = (blockIdx.x % nkt) * tkx;
    cplx<T> *base = spec + (size_t)k * ny * sk + x0;
    for (int e = threadIdx.x; e < ny * tkx; e += blockDim.x) {
        const int j = e / tkx, l = e - j * tkx;
        A[e] = base[(size_t)j * sk + l];
    }
    __syncthreads();
    const cplx<T> *R = fft_lines<T, SIGN>(A, B, tkx, 1, tkx, fp, twy, true);
    for (int e = threadIdx.x; e < ny * tkx; e += blockDim.x) {
        const int j = e / tkx, l = e - j * tkx;
        base[(size_t)j * sk + l] = R[e];
    }
}

template <typename T> struct PoissonMat {
    const T *idz, *ihc, *lam;
    int nz, walls;
    FSEI_D T a(int i) const { return (walls && i == 0) ? T(0) : ihc[i] * idz[i]; }
    FSEI_D T c(int i) const { return (walls && i == nz - 1) ? T(0) : ihc[i + 1] * idz[i]; }
    FSEI_D T b(int l, int i) const { return -(a(i) + c(i)) - lam[l]; }
};

template <typename T>
__global__ void __launch_bounds__(512)
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
    for (int e = threadIdx.x; e < nz * tkx; e += blockDim.x) {
        const int k = e / tkx, l = e - k * tkx;
        D[e] = base[(size_t)k * plane + l];
    }
    __syncthreads();
    PoissonMat<T> M{Metric<T>::idz(g), Metric<T>::ihc(g), lam, nz, g.walls};
    tri_fly_solve<T>(D, tkx, 1, fa, fc, tkx, 1, tkx, nz, P, !g.walls, M, rr, rlo, rdi, rup, rs);
    // modes solved exactly in double (k_poisson_exact, launched before this
    // kernel) keep their values
    const unsigned char *ex = exact + (size_t)ky * sk + x0;
    for (int e = threadIdx.x; e < nz * tkx; e += blockDim.x) {
        const int k = e / tkx, l = e - k * tkx;
        if (!ex[l]) base[(size_t)k * plane + l] = scale * D[e];
    }
}

// Thomas' algorithm in double on one z line held in shared memory (one
// thread).  With pin0 the unknown at k = 0 is fixed to 0 and rows 1..nz-1
// are solved; a periodic line without pin0 is solved with Sherman-Morrison.
// yr, yi: the right-hand side on entry, the solution on exit; cp, zz:
// scratch of nz doubles.
FSEI_D void exact_line(const GridDev &g, double lam, bool pin0, double *yr, double *yi,
                       double *cp, double *zz) {
    const int nz = g.nz;
    const bool walls = g.walls != 0;
    const int k0 = pin0 ? 1 : 0;
    const bool cyc = !walls && !pin0;
    auto A = [&](int k) { return (walls && k == 0) ? 0.0 : g.ihc[k] * g.idz[k]; };
    auto C = [&](int k) { return (walls && k == nz - 1) ? 0.0 : g.ihc[k + 1] * g.idz[k]; };
    const double gsm = cyc ? (A(0) + C(0)) + lam : 0.0;   // -b_0
    auto Bm = [&](int k) {
        double b = -(A(k) + C(k)) - lam;
        if (cyc && k == 0) b -= gsm;
        if (cyc && k == nz - 1) b -= C(nz - 1) * A(0) / gsm;
        return b;
    };
    double inv = 1.0 / Bm(k0);
    cp[k0] = C(k0) * inv;
    yr[k0] *= inv;
    yi[k0] *= inv;
    zz[k0] = cyc ? gsm * inv : 0.0;
    for (int k = k0 + 1; k < nz; ++k) {
        const double a = A(k);
        inv = 1.0 / (Bm(k) - a * cp[k - 1]);
        cp[k] = C(k) * inv;
        yr[k] = (yr[k] - a * yr[k - 1]) * inv;
        yi[k] = (yi[k] - a * yi[k - 1]) * inv;
        if (cyc) zz[k] = ((k == nz - 1 ? C(nz - 1) : 0.0) - a * zz[k - 1]) * inv;
    }
    for (int k = nz - 2; k >= k0; --k) {
        yr[k] -= cp[k] * yr[k + 1];
        yi[k] -= cp[k] * yi[k + 1];
        if (cyc) zz[k] -= cp[k] * zz[k + 1];
    }
    if (cyc) {
        const double vl = A(0) / gsm;
        const double fac = 1.0 / (1.0 + zz[0] + vl * zz[nz - 1]);
        const double fr = (yr[0] + vl * yr[nz - 1]) * fac;
        const double fi = (yi[0] + vl * yi[nz - 1]) * fac;
        for (int k = 0; k < nz; ++k) {
            yr[k] -= fr * zz[k];
            yi[k] -= fi * zz[k];
        }
    }
    if (pin0) {
        yr[0] = 0.0;
        yi[0] = 0.0;
    }
}

// One block per exactly solved mode: the z line is staged in shared memory
// (double), solved by one thread, written back scaled by 1/(nx ny).  For the
// (0, 0) mode the volume-weighted mean is removed afterwards (gauge); with
// compat the right-hand side of that mode first loses its own dz-weighted
// mean (makes an arbitrary right-hand side compatible).
template <typename T>
__global__ void __launch_bounds__(128)
k_poisson_exact(GridDev g, cplx<T> *spec, const int *modes, const double *lamx,
                const double *lamy, double scale, int compat) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nz = g.nz;
    double *yr = reinterpret_cast<double *>(smraw);
    double *yi = yr + nz, *cp = yi + nz, *zz = cp + nz;
    __shared__ double red[2][128];
    const int code = modes[blockIdx.x];
    const int kx = code % g.sk, ky = code / g.sk;
    const bool zero_mode = kx == 0 && ky == 0;
    const size_t stride = (size_t)g.ny * g.sk;
    cplx<T> *line = spec + (size_t)ky * g.sk + kx;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        const cplx<T> v = line[(size_t)k * stride];
        yr[k] = (double)v.re;
        yi[k] = (double)v.im;
    }
    __syncthreads();
    // dz-weighted means of the line (before: compat; after: gauge)
    auto wmean = [&](double &mr, double &mi) {
        double sr = 0.0, si = 0.0;
        for (int k = threadIdx.x; k < nz; k += blockDim.x) {
            sr += yr[k] * g.dz[k];
            si += yi[k] * g.dz[k];
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
        for (int k = threadIdx.x; k < nz; k += blockDim.x) { yr[k] -= mr; yi[k] -= mi; }
        __syncthreads();
    }
    if (threadIdx.x == 0) exact_line(g, lamx[kx] + lamy[ky], zero_mode, yr, yi, cp, zz);
    __syncthreads();
    double mr = 0.0, mi = 0.0;
    if (zero_mode) wmean(mr, mi);
    for (int k = threadIdx.x; k < nz; k += blockDim.x)
        line[(size_t)k * stride] = cplx<T>{T((yr[k] - mr) * scale), T((yi[k] - mi) * scale)};
}

template <typename T>
__global__ void __launch_bounds__(512)
k_irfft_x(GridDev g, const cplx<T> *__restrict__ spec, T *__restrict__ dst,
          const cplx<T> *__restrict__ twx, const cplx<T> *__restrict__ twpost, FftPlanDev fp,
          int ry) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nx = g.nx, ny = g.ny, mx = g.mx, sk = g.sk;
    const int ls = mx | 1;
    cplx<T> *A = reinterpret_cast<cplx<T> *>(smraw);
    cplx<T> *B = A + (size_t)ry * ls;
    const int nby = ny / ry;
    const int k = blockIdx.x / nby, j0 = (blockIdx.x % nby) * ry;
    for (int e = threadIdx.x; e < ry * mx; e += blockDim.x) {
        const int r = e / mx, kx = e - r * mx;
        const cplx<T> *row = spec + ((size_t)k * ny + j0 + r) * sk;
        const cplx<T> xk = row[kx];
        const cplx<T> xm = conj(row[mx - kx]);
        const cplx<T> ev = xk + xm;
        const cplx<T> od = (xk - xm) * conj(twpost[kx]);
        A[r * ls + kx] = ev + mul_i<T, 1>(od);
    }
    __syncthreads();
    const cplx<T> *R = fft_lines<T, 1>(A, B, 1, ls, ry, fp, twx, false);
    for (int e = threadIdx.x; e < ry * nx; e += blockDim.x) {
        const int r = e / nx, i = e - r * nx;
        dst[fid(i, j0 + r, k, nx, ny)] = reinterpret_cast<const T *>(R + (size_t)r * ls)[i];
    }
}

}  // namespace

template <typename T> size_t smem_fft_x(const GridDev &g, const Work<T> &W) {
    return 2 * sizeof(cplx<T>) * (size_t)W.ry * (g.mx | 1);
}
template <typename T> size_t smem_fft_y(const GridDev &g, const Work<T> &W) {
    return 2 * sizeof(cplx<T>) * (size_t)W.tkx * g.ny;
}
template <typename T> size_t smem_poisson(const GridDev &g, const Work<T> &W) {
    const size_t rs = 2 * W.pz_poisson + 1;
    return sizeof(cplx<T>) * ((size_t)g.nz * W.tkx + W.tkx * rs) +
           sizeof(T) * (2 * (size_t)g.nz * W.tkx + 3 * W.tkx * rs + W.tkx);
}

template <typename T> void launch_rfft_x(const GridDev &g, Work<T> &W, const StepScalars *sc,
                                         const T *src, int mode, cudaStream_t st) {
    const int blocks = g.nz * (g.ny / W.ry);
    const int threads = 256;
    if (mode == 0)
        k_rfft_x<T, 0><<<blocks, threads, smem_fft_x(g, W), st>>>(
            g, W.q0, W.q1, W.q2, nullptr, W.spec, W.twx, W.twpost, W.fpx, sc, W.ry);
    else
        k_rfft_x<T, 1><<<blocks, threads, smem_fft_x(g, W), st>>>(
            g, nullptr, nullptr, nullptr, src, W.spec, W.twx, W.twpost, W.fpx, sc, W.ry);
}

template <typename T> void launch_fft_y(const GridDev &g, Work<T> &W, int inverse, cudaStream_t st) {
    const int blocks = g.nz * (g.sk / W.tkx);
    if (inverse)
        k_fft_y<T, 1><<<blocks, 256, smem_fft_y(g, W), st>>>(g, W.spec, W.twy, W.fpy, W.tkx);
    else
        k_fft_y<T, -1><<<blocks, 256, smem_fft_y(g, W), st>>>(g, W.spec, W.twy, W.fpy, W.tkx);
}

template <typename T> void launch_poisson_z(const GridDev &g, Work<T> &W, cudaStream_t st) {
    const int blocks = g.ny * (g.sk / W.tkx);
    const int threads = ((W.tkx * W.pz_poisson + 31) / 32) * 32;
    const double scale = 1.0 / ((double)g.nx * g.ny);
    // exact modes first: they read the untouched right-hand side
    k_poisson_exact<T><<<W.n_nzm, 128, 4 * sizeof(double) * g.nz, st>>>(
        g, W.spec, W.nzm, W.lamx_d, W.lamy_d, scale, 0);
    k_poisson_z<T><<<blocks, threads, smem_poisson(g, W), st>>>(
        g, W.spec, W.lamx, W.lamy, W.exact, W.tkx, W.pz_poisson, T(scale));
}

template <typename T> void launch_irfft_x(const GridDev &g, Work<T> &W, T *dst, cudaStream_t st) {
    const int blocks = g.nz * (g.ny / W.ry);
    k_irfft_x<T><<<blocks, 256, smem_fft_x(g, W), st>>>(g, W.spec, dst, W.twx, W.twpost, W.fpx,
                                                        W.ry);
}

template <typename T> void set_smem_limits_poisson(const GridDev &g, const Work<T> &W) {
    cudaFuncSetAttribute(k_rfft_x<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem_fft_x(g, W));
    cudaFuncSetAttribute(k_rfft_x<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem_fft_x(g, W));
    cudaFuncSetAttribute(k_irfft_x<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem_fft_x(g, W));
    cudaFuncSetAttribute(k_fft_y<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem_fft_y(g, W));
    cudaFuncSetAttribute(k_fft_y<T, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem_fft_y(g, W));
    cudaFuncSetAttribute(k_poisson_z<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem_poisson(g, W));
    cudaFuncSetAttribute(k_poisson_exact<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(4 * sizeof(double) * g.nz));
}

#define FSEI_INST(T)                                                                           \
    template size_t smem_fft_x<T>(const GridDev &, const Work<T> &);                          \
    template size_t smem_fft_y<T>(const GridDev &, const Work<T> &);                          \
    template size_t smem_poisson<T>(const GridDev &, const Work<T> &);                        \
    template void launch_rfft_x<T>(const GridDev &, Work<T> &, const StepScalars *, const T *, \
                                   int, cudaStream_t);                                        \
    template void launch_fft_y<T>(const GridDev &, Work<T> &, int, cudaStream_t);              \
    template void launch_poisson_z<T>(const GridDev &, Work<T> &, cudaStream_t);               \
    template void launch_irfft_x<T>(const GridDev &, Work<T> &, T *, cudaStream_t);            \
    template void set_smem_limits_poisson<T>(const GridDev &, const Work<T> &);
FSEI_INST(float)
FSEI_INST(double)
#undef FSEI_INST

}  // namespace fsei
