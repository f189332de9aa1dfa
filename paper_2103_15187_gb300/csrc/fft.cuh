// Batched complex FFTs in shared memory for the pressure Poisson solve
// (Fourier transform in the two periodic directions, Sec. 3.1 / Sec. 4; the
// paper uses FFTW3 on the CPU, here every transform is hand-written).
//
// Self-sorting mixed-radix Stockham transform of length N = 2^a 3^b.  A pass
// of radix R with p = product of the radices already applied takes, for
// each butterfly index i < N/R (k = i mod p), the inputs x_r = in[i + r N/R],
// multiplies x_r by w^(r k N / (p R)) with w = exp(-2 pi i / N) (conjugated
// for the inverse), applies the length-R DFT, and stores output r at
// out[(i - k) R + k + r p].  After the last pass the result is in natural
// order.  Forward transforms are unnormalised sums with exp(-...); inverse
// ones unnormalised sums with exp(+...).
#pragma once
#include "common.cuh"

namespace fsei {

struct FftPlanDev {
    int n;        // transform length
    int nr;       // number of passes
    int rad[16];  // radix of each pass (2, 3 or 4)
};

template <typename T, int SIGN>
FSEI_D void dft2(cplx<T> &x0, cplx<T> &x1) {
    const cplx<T> a = x0 + x1, b = x0 - x1;
    x0 = a;
    x1 = b;
}

template <typename T, int SIGN>
FSEI_D void dft3(cplx<T> &x0, cplx<T> &x1, cplx<T> &x2) {
    const T h = T(0.86602540378443864676);   // sqrt(3)/2
    const cplx<T> t = x1 + x2;
    const cplx<T> m = x0 - T(0.5) * t;
    const cplx<T> dd = mul_i<T, SIGN>(h * (x1 - x2));
    x0 = x0 + t;
    x1 = m + dd;
    x2 = m - dd;
}

template <typename T, int SIGN>
FSEI_D void dft4(cplx<T> &x0, cplx<T> &x1, cplx<T> &x2, cplx<T> &x3) {
    const cplx<T> a = x0 + x2, b = x0 - x2, c = x1 + x3;
    const cplx<T> d = mul_i<T, SIGN>(x1 - x3);
    x0 = a + c;
    x2 = a - c;
    x1 = b + d;
    x3 = b - d;
}

// Transform nl lines.  Element i of line l: buf[i * es + l * ls].  Data
// starts in a; b is scratch of the same size.  Returns the buffer holding
// the result.  tw: table of w^m, m < N (forward sign), normally staged in
// shared memory by the caller.  Must be called by every thread of the block;
// ends with a barrier.
template <typename T, int SIGN>
__device__ cplx<T> *fft_lines(cplx<T> *a, cplx<T> *b, int es, int ls, int nl,
                              const FftPlanDev &fp, const cplx<T> *__restrict__ tw,
                              bool line_fastest) {
    const int N = fp.n;
    // the radices packed two bits each (radix - 2): a run-time index into
    // fp.rad would place the plan in local memory
    unsigned code = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q)
        if (q < fp.nr) code |= (unsigned)(fp.rad[q] - 2) << (2 * q);
    int p = 1;
    cplx<T> *src = a, *dst = b;
    for (int s = 0; s < fp.nr; ++s) {
        const int R = (int)((code >> (2 * s)) & 3u) + 2;
        const int TN = N / R;
        const int tstep = N / (p * R);
        const int total = nl * TN;
        for (int w = threadIdx.x; w < total; w += blockDim.x) {
            int l, i;
            if (line_fastest) { i = ddiv(w, nl); l = w - i * nl; }
            else { l = ddiv(w, TN); i = w - l * TN; }
            const int k = dmod(i, p);
            const int j = (i - k) * R + k;
            cplx<T> x[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (r < R) {
                    cplx<T> v = src[(i + r * TN) * es + l * ls];
                    if (r > 0 && k > 0) {
                        cplx<T> wv = tw[r * k * tstep];
                        if (SIGN > 0) wv = conj(wv);
                        v = v * wv;
                    }
                    x[r] = v;
                }
            }
            if (R == 4) dft4<T, SIGN>(x[0], x[1], x[2], x[3]);
            else if (R == 2) dft2<T, SIGN>(x[0], x[1]);
            else dft3<T, SIGN>(x[0], x[1], x[2]);
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (r < R) dst[(j + r * p) * es + l * ls] = x[r];
        }
        __syncthreads();
        cplx<T> *tmp = src;
        src = dst;
        dst = tmp;
        p *= R;
    }
    return src;
}

// In-register DFT of length B: a power of two (B <= 32), iterative radix-2
// with bit-reversed input order, every index a compile-time constant once
// unrolled; 3; or 3 M with M a power of two (M DFTs of the residues n mod
// 3, the twiddles w_B^(r k'), then DFTs of length 3).  tw: table of w^m =
// exp(-2 pi i m / N), m < N, for a transform length N that B divides (stage
// twiddles are tw[k N / (2h)], w_3 = tw[N / 3], w_B^j = tw[j N / B]).
template <int B> struct Log2 { static constexpr int v = 1 + Log2<B / 2>::v; };
template <> struct Log2<1> { static constexpr int v = 0; };

template <typename T, int B, int SIGN>
FSEI_D void dft_reg(cplx<T> (&x)[B], const cplx<T> *tw, int N) {
    if constexpr (B == 3) {
        // y1 = x0 + w x1 + w* x2, y2 = x0 + w* x1 + w x2 (w^2 = w*)
        cplx<T> w = tw[N / 3];
        if (SIGN > 0) w = conj(w);
        const cplx<T> s = x[1] + x[2], d = x[1] - x[2];
        const cplx<T> m{x[0].re + w.re * s.re, x[0].im + w.re * s.im};
        const cplx<T> j{-w.im * d.im, w.im * d.re};   // i w.im d
        x[0] = x[0] + s;
        x[1] = m + j;
        x[2] = m - j;
    } else if constexpr (B % 3 == 0) {
        constexpr int M = B / 3;
        cplx<T> y[3][M];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
#pragma unroll
            for (int m = 0; m < M; ++m) y[r][m] = x[3 * m + r];
            dft_reg<T, M, SIGN>(y[r], tw, N);
        }
#pragma unroll
        for (int kp = 0; kp < M; ++kp) {
            cplx<T> z[3];
            z[0] = y[0][kp];
#pragma unroll
            for (int r = 1; r < 3; ++r) {
                cplx<T> w = tw[(N / B) * r * kp];
                if (SIGN > 0) w = conj(w);
                z[r] = kp == 0 ? y[r][kp] : y[r][kp] * w;
            }
            dft_reg<T, 3, SIGN>(z, tw, N);
#pragma unroll
            for (int q = 0; q < 3; ++q) x[kp + M * q] = z[q];
        }
    } else {
        constexpr int LB = Log2<B>::v;
#pragma unroll
        for (int i = 0; i < B; ++i) {
            int r = 0;
#pragma unroll
            for (int b = 0; b < LB; ++b) r |= ((i >> b) & 1) << (LB - 1 - b);
            if (r > i) {
                const cplx<T> t = x[i];
                x[i] = x[r];
                x[r] = t;
            }
        }
#pragma unroll
        for (int h = 1; h < B; h *= 2) {
#pragma unroll
            for (int g0 = 0; g0 < B; g0 += 2 * h) {
#pragma unroll
                for (int k = 0; k < h; ++k) {
                    cplx<T> w = tw[k * (N / (2 * h))];
                    if (SIGN > 0) w = conj(w);
                    const cplx<T> a = x[g0 + k];
                    const cplx<T> b = (k == 0) ? x[g0 + k + h] : x[g0 + k + h] * w;
                    x[g0 + k] = a + b;
                    x[g0 + k + h] = a - b;
                }
            }
        }
    }
}

// Split N = N1 N2 of the two-pass transforms (N1 >= N2; N1 <= 32 and N2 <=
// 24 so that the register arrays stay small; each a power of two, 3, or 3
// times a power of two), 0 for lengths that take the Stockham passes of
// fft_lines.  The shared-memory two-pass of fft_lines_fast (the forward x
// transform) takes the powers of two up to 256 only: every length it lists
// is compiled into each kernel that calls it, and more cases there cost
// those kernels registers; the y transforms (k_fft_y_2p) and the inverse x
// transform (k_irfft_x_2p, up to 256) are instantiated per split.
FSEI_HD int fft_split_n1(int n) {
    switch (n) {
    case 12: return 4;
    case 16: return 4;
    case 24: return 6;
    case 32: return 8;
    case 48: return 8;
    case 64: return 8;
    case 96: return 12;
    case 128: return 16;
    case 192: return 16;
    case 256: return 16;
    case 384: return 24;
    case 512: return 32;
    default: return 0;
    }
}
// Complex values of scratch per line that the two-pass transform of a line
// stored whole (element stride 1) needs: N2 blocks of N1 + 1 (the padding
// staggers the banks of the transposed accesses); n otherwise.
FSEI_HD int fft_scratch_len(int n) {
    const int n1 = fft_split_n1(n);
    return n1 ? (n / n1) * (n1 + 1) : n;
}

// Two-pass transform of nl lines of length N = N1 N2, with n = N2 n1 + n2
// and k = k1 + N1 k2:
//   X[k] = sum_n2 w_N2^(n2 k2) w_N^(n2 k1) sum_n1 w_N1^(n1 k1) x[N2 n1 + n2].
// Pass 1, item (l, n2): the N1 values x[N2 n1 + n2] of line l, an in-register
// DFT of length N1, the twiddles w_N^(n2 k1), stored to b.  Pass 2, item
// (l, k1): the N2 values of k1 from b, an in-register DFT of length N2,
// X[k1 + N1 k2] to a.  LF (lines fastest, the layout of a with element
// stride es, line stride ls): b has a's layout, value (n2, k1) at position
// n2 N1 + k1; otherwise (lines stored whole) line l's values sit in b at
// l bls + n2 (N1 + 1) + k1.  tw: w^m = exp(-2 pi i m / N), m < N (conjugated
// for SIGN > 0).  Every thread of the block calls it; returns a (natural
// order) after a barrier.
template <typename T, int SIGN, int N1, int N2, bool LF>
__device__ cplx<T> *fft_lines_2p(cplx<T> *a, cplx<T> *b, int es, int ls, int bls, int nl,
                                 const cplx<T> *__restrict__ tw) {
    constexpr int N = N1 * N2;
    for (int w = threadIdx.x; w < nl * N2; w += blockDim.x) {
        int l, n2;
        if (LF) { n2 = ddiv(w, nl); l = w - n2 * nl; }
        else { l = w / N2; n2 = w - l * N2; }
        cplx<T> x[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) x[n1] = a[(n1 * N2 + n2) * es + l * ls];
        dft_reg<T, N1, SIGN>(x, tw, N);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) {
            cplx<T> t = tw[n2 * k1];
            if (SIGN > 0) t = conj(t);
            x[k1] = x[k1] * t;
        }
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            if (LF) b[(n2 * N1 + k1) * es + l * ls] = x[k1];
            else b[l * bls + n2 * (N1 + 1) + k1] = x[k1];
        }
    }
    __syncthreads();
    for (int w = threadIdx.x; w < nl * N1; w += blockDim.x) {
        int l, k1;
        if (LF) { k1 = ddiv(w, nl); l = w - k1 * nl; }
        else { l = w / N1; k1 = w - l * N1; }
        cplx<T> y[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2)
            y[n2] = LF ? b[(n2 * N1 + k1) * es + l * ls] : b[l * bls + n2 * (N1 + 1) + k1];
        dft_reg<T, N2, SIGN>(y, tw, N);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) a[(k1 + N1 * k2) * es + l * ls] = y[k2];
    }
    __syncthreads();
    return a;
}

// fft_lines with the two-pass transform for the lengths fft_split_n1 lists;
// b then holds at least nl fft_scratch_len(N) values (lines stored whole,
// line stride bls in b) or a's layout (LF).
template <typename T, int SIGN, bool LF>
__device__ cplx<T> *fft_lines_fast(cplx<T> *a, cplx<T> *b, int es, int ls, int bls, int nl,
                                   const FftPlanDev &fp, const cplx<T> *__restrict__ tw) {
    switch (fp.n) {
    case 16: return fft_lines_2p<T, SIGN, 4, 4, LF>(a, b, es, ls, bls, nl, tw);
    case 32: return fft_lines_2p<T, SIGN, 8, 4, LF>(a, b, es, ls, bls, nl, tw);
    case 64: return fft_lines_2p<T, SIGN, 8, 8, LF>(a, b, es, ls, bls, nl, tw);
    case 128: return fft_lines_2p<T, SIGN, 16, 8, LF>(a, b, es, ls, bls, nl, tw);
    case 256: return fft_lines_2p<T, SIGN, 16, 16, LF>(a, b, es, ls, bls, nl, tw);
    default: return fft_lines<T, SIGN>(a, b, es, ls, nl, fp, tw, LF);
    }
}

}  // namespace fsei
