// Immersed-boundary forcing by moving least squares (Sec. 2.1, Eq. 4;
// Sec. 3.2) and the hydrodynamic loads on the immersed surface (Eqs. 5-7).
//
//   k_ib_force   one warp per (marker, velocity component): lane k < 27
//                holds support node k of the 3 x 3 x 3 nodes of that
//                component's staggered grid nearest to the marker; the
//                moment matrix A = sum_k w_k p_k p_k^T (10 distinct entries)
//                by warp reductions, A alpha = p(x_b) solved by every lane
//                (4 x 4, double), the transfer operators phi_k = w_k p_k .
//                alpha, the interpolated velocity by a reduction, the direct
//                force F = (U_b - u(x_b)) / dt, spread with atomic adds of
//                phi_k F dV_b / dV_k.
//   k_ib_loads   one warp per face: at the probe x_f + h n_f (and x_f - h n_f
//                for a two-sided face) the same fit of p (value) and of u, v,
//                w (linear coefficients = gradient); traction -p n + tau . n,
//                tau = Re^-1 (grad u + grad u^T); face load times the area,
//                a third of it added to each of the face's nodes.
//
// Readings (where the paper defers to its citations): the support centred on
// the nearest node (a point exactly halfway between two nodes takes the one
// whose half-open control volume [lower, upper) holds it); weight exp(-r^2), r
// the node offset over the nearest node's control extents (dx, dy; dz_k for
// centre points, hc_k for w faces); basis [1, x, y, z] centred and scaled at
// the evaluation point; dV_k = dx dy dz_k (u, v) or dx dy hc_k (w).  A support
// that would leave the interior z nodes of a walled grid skips its marker
// (face) and counts it.  The fits run in double whatever the field type.
#include "kernels.cuh"

namespace fsei {

namespace {

enum { LOC_U = 0, LOC_V = 1, LOC_W = 2, LOC_P = 3 };

FSEI_D double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// nearest node index along a uniform periodic axis of n nodes at
// (i + off) h, and the offset of node c + d from x (x taken into [0, n h))
FSEI_D void axis_uniform(double x, double h, double off, int n, int d, int &idx, double &rel) {
    const double len = n * h;
    x -= floor(x / len) * len;
    const int c = (int)floor(x / h - off + 0.5);
    rel = ((c + d) + off) * h - x;
    idx = ((c + d) % n + n) % n;
}

// One lane's support node of point x for component loc and the fit data:
// returns false (for every lane) when the support leaves the interior z
// nodes of a walled grid.  s: the node offset over the extents h; hz: the
// z extent; vol: the node's control volume.
FSEI_D bool support_node(const GridDev &g, int loc, const double x[3], int lane, size_t &cell,
                         double s[3], double h[3], double &vol) {
    const int di = lane % 3 - 1, dj = (lane / 3) % 3 - 1, dk = lane / 9 - 1;
    int ix, iy, iz;
    double rx, ry, rz;
    axis_uniform(x[0], g.dx, loc == LOC_U ? 0.0 : 0.5, g.nx, di, ix, rx);
    axis_uniform(x[1], g.dy, loc == LOC_V ? 0.0 : 0.5, g.ny, dj, iy, ry);
    // z: the cell holding z (binary search over the faces), then the nearest
    // face or centre
    const int nz = g.nz;
    const double z0 = g.zf[0], lz = g.zf[nz] - z0;
    double z = x[2];
    if (!g.walls) z = z0 + (z - z0 - floor((z - z0) / lz) * lz);
    int lo = 0, hi = nz - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g.zf[mid] <= z) lo = mid;
        else hi = mid - 1;
    }
    int c;
    if (loc == LOC_W) {
        // a tie (z on the centre between the two faces) goes to the upper
        // face, whose control volume [zc_lo, zc_lo+1) holds z
        c = (z - g.zf[lo] < g.zf[lo + 1] - z) ? lo : lo + 1;
    } else {
        c = lo;
        const double zc = 0.5 * (g.zf[lo] + g.zf[lo + 1]);
        if (z < zc && lo > 0 && zc - z > z - 0.5 * (g.zf[lo - 1] + g.zf[lo])) c = lo - 1;
        if (z > zc && lo < nz - 1 && z - zc > 0.5 * (g.zf[lo + 1] + g.zf[lo + 2]) - z) c = lo + 1;
    }
    if (g.walls) {
        const int first = loc == LOC_W ? 2 : 1;
        if (c < first || c > nz - 2) return false;
    }
    int kk = c + dk;
    double shift = 0.0;
    if (!g.walls) {
        if (kk < 0) { kk += nz; shift = -lz; }
        if (kk >= nz) { kk -= nz; shift = lz; }
        if (c == nz && loc == LOC_W) { c = 0; }   // the top face is face 0
    }
    const double zn = loc == LOC_W ? g.zf[kk] : 0.5 * (g.zf[kk] + g.zf[kk + 1]);
    rz = zn + shift - z;
    iz = kk;
    // extents of the nearest node (c, wrapped) and this node's volume
    const int cw = (c % nz + nz) % nz;
    h[0] = g.dx;
    h[1] = g.dy;
    h[2] = loc == LOC_W ? 1.0 / g.ihc[cw] : g.dz[cw];
    s[0] = rx / h[0];
    s[1] = ry / h[1];
    s[2] = rz / h[2];
    vol = g.dx * g.dy * (loc == LOC_W ? 1.0 / g.ihc[iz] : g.dz[iz]);
    cell = ((size_t)iz * g.ny + iy) * g.nx + ix;
    return true;
}

// Solve the symmetric positive definite 4 x 4 system A y = b (A given by its
// 10 distinct entries a00 a01 a02 a03 a11 a12 a13 a22 a23 a33) by Cholesky.
FSEI_D void spd4_solve(const double a[10], double b[4]) {
    double l00 = sqrt(a[0]);
    double l10 = a[1] / l00, l20 = a[2] / l00, l30 = a[3] / l00;
    double l11 = sqrt(a[4] - l10 * l10);
    double l21 = (a[5] - l20 * l10) / l11, l31 = (a[6] - l30 * l10) / l11;
    double l22 = sqrt(a[7] - l20 * l20 - l21 * l21);
    double l32 = (a[8] - l30 * l20 - l31 * l21) / l22;
    double l33 = sqrt(a[9] - l30 * l30 - l31 * l31 - l32 * l32);
    // forward L y = b, then L^T x = y
    const double y0 = b[0] / l00;
    const double y1 = (b[1] - l10 * y0) / l11;
    const double y2 = (b[2] - l20 * y0 - l21 * y1) / l22;
    const double y3 = (b[3] - l30 * y0 - l31 * y1 - l32 * y2) / l33;
    b[3] = y3 / l33;
    b[2] = (y2 - l32 * b[3]) / l22;
    b[1] = (y1 - l21 * b[2] - l31 * b[3]) / l11;
    b[0] = (y0 - l10 * b[1] - l20 * b[2] - l30 * b[3]) / l00;
}

// moment matrix of the lane's weighted basis row (lanes >= 27 add nothing)
FSEI_D void moments(bool on, double w, const double p[4], double a[10]) {
    int m = 0;
    for (int i = 0; i < 4; ++i)
        for (int j = i; j < 4; ++j) a[m++] = warp_sum(on ? w * p[i] * p[j] : 0.0);
}

}  // namespace

// One warp per (marker, component); markers b = warp / 3.
template <typename T>
__global__ void __launch_bounds__(256)
k_ib_force(GridDev g, const T *__restrict__ u, const T *__restrict__ v, const T *__restrict__ w,
           const double *__restrict__ xb, const double *__restrict__ ub,
           const double *__restrict__ dvb, int nm, double dt, T *fx, T *fy, T *fz,
           double *u_at, int *skipped) {
    const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= 3 * nm) return;
    const int b = warp / 3, comp = warp - 3 * b;
    const double x[3] = {xb[3 * b], xb[3 * b + 1], xb[3 * b + 2]};
    size_t cell = 0;
    double s[3], h[3], vol = 1.0;
    const bool ok = support_node(g, comp, x, lane < 27 ? lane : 13, cell, s, h, vol);
    if (!ok) {
        if (lane == 0) {
            atomicAdd(skipped, 1);
            if (u_at) u_at[3 * b + comp] = 0.0;
        }
        return;
    }
    const bool on = lane < 27;
    const double wk = on ? exp(-(s[0] * s[0] + s[1] * s[1] + s[2] * s[2])) : 0.0;
    const double p[4] = {1.0, s[0], s[1], s[2]};
    double a[10];
    moments(on, wk, p, a);
    double alpha[4] = {1.0, 0.0, 0.0, 0.0};
    spd4_solve(a, alpha);
    const double phi = on ? wk * (p[0] * alpha[0] + p[1] * alpha[1] + p[2] * alpha[2] +
                                  p[3] * alpha[3])
                          : 0.0;
    const T *fld = comp == 0 ? u : (comp == 1 ? v : w);
    const double val = warp_sum(on ? phi * (double)fld[cell] : 0.0);
    const double F = (ub[3 * b + comp] - val) / dt;
    T *fo = comp == 0 ? fx : (comp == 1 ? fy : fz);
    if (on) atomicAdd(fo + cell, T(phi * F * dvb[b] / vol));
    if (lane == 0 && u_at) u_at[3 * b + comp] = val;
}

namespace {

// value and gradient of the fit of field f (location loc) at x, in every
// lane; false if the support leaves the interior
template <typename T>
FSEI_D bool fit_at(const GridDev &g, int loc, const T *f, const double x[3], double &val,
                   double grad[3]) {
    const int lane = threadIdx.x & 31;
    size_t cell = 0;
    double s[3], h[3], vol;
    if (!support_node(g, loc, x, lane < 27 ? lane : 13, cell, s, h, vol)) return false;
    const bool on = lane < 27;
    const double wk = on ? exp(-(s[0] * s[0] + s[1] * s[1] + s[2] * s[2])) : 0.0;
    const double p[4] = {1.0, s[0], s[1], s[2]};
    double a[10];
    moments(on, wk, p, a);
    const double fv = on ? (double)f[cell] : 0.0;
    double c[4];
    for (int i = 0; i < 4; ++i) c[i] = warp_sum(on ? wk * p[i] * fv : 0.0);
    spd4_solve(a, c);
    val = c[0];
    grad[0] = c[1] / h[0];
    grad[1] = c[2] / h[1];
    grad[2] = c[3] / h[2];
    return true;
}

}  // namespace

// One warp per face.
template <typename T>
__global__ void __launch_bounds__(256)
k_ib_loads(GridDev g, const T *__restrict__ p, const T *__restrict__ u, const T *__restrict__ v,
           const T *__restrict__ w, const double *__restrict__ xf, const double *__restrict__ nf,
           const double *__restrict__ af, const int *__restrict__ two_sided,
           const int *__restrict__ tris, int nfaces, int nnodes, double probe, double inv_re,
           double *face_force, double *node_force, int *skipped) {
    const int f = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (f >= nfaces) return;
    const double n[3] = {nf[3 * f], nf[3 * f + 1], nf[3 * f + 2]};
    const int sides = (two_sided && two_sided[f]) ? 2 : 1;
    double t[3] = {0.0, 0.0, 0.0};
    bool ok = true;
    for (int side = 0; side < sides && ok; ++side) {
        const double sg = side == 0 ? 1.0 : -1.0;
        const double x[3] = {xf[3 * f] + sg * probe * n[0], xf[3 * f + 1] + sg * probe * n[1],
                             xf[3 * f + 2] + sg * probe * n[2]};
        double pv, gp[3], gr[3][3], val;
        ok = fit_at(g, LOC_P, p, x, pv, gp) && fit_at(g, LOC_U, u, x, val, gr[0]) &&
             fit_at(g, LOC_V, v, x, val, gr[1]) && fit_at(g, LOC_W, w, x, val, gr[2]);
        if (!ok) break;
        for (int i = 0; i < 3; ++i) {
            double tn = 0.0;
            for (int j = 0; j < 3; ++j) tn += (gr[i][j] + gr[j][i]) * n[j];
            t[i] += sg * (-pv * n[i] + inv_re * tn);
        }
    }
    if (!ok) {
        if (lane == 0) {
            atomicAdd(skipped, 1);
            for (int i = 0; i < 3; ++i) face_force[3 * f + i] = 0.0;
        }
        return;
    }
    if (lane < 3) {
        const double F = t[lane] * af[f];
        face_force[3 * f + lane] = F;
        if (node_force && tris)
            for (int q = 0; q < 3; ++q) {
                const int node = tris[3 * f + q];
                if (node >= 0 && node < nnodes)
                    atomicAdd(node_force + 3 * (size_t)node + lane, F / 3.0);
                else if (lane == 0)
                    atomicAdd(skipped + 1, 1);   // a node index outside the node list
            }
    }
}

template <typename T>
void launch_ib_force(const GridDev &g, const T *u, const T *v, const T *w, const double *xb,
                     const double *ub, const double *dvb, int nm, double dt, T *fx, T *fy,
                     T *fz, double *u_at, int *skipped, cudaStream_t st) {
    if (nm <= 0) return;
    const long long warps = 3LL * nm;
    const int blocks = (int)((warps * 32 + 255) / 256);
    k_ib_force<T><<<blocks, 256, 0, st>>>(g, u, v, w, xb, ub, dvb, nm, dt, fx, fy, fz, u_at,
                                          skipped);
}

template <typename T>
void launch_ib_loads(const GridDev &g, const T *p, const T *u, const T *v, const T *w,
                     const double *xf, const double *nf, const double *af, const int *two_sided,
                     const int *tris, int nfaces, int nnodes, double probe, double inv_re,
                     double *face_force, double *node_force, int *skipped, cudaStream_t st) {
    if (nfaces <= 0) return;
    const int blocks = (int)(((long long)nfaces * 32 + 255) / 256);
    k_ib_loads<T><<<blocks, 256, 0, st>>>(g, p, u, v, w, xf, nf, af, two_sided, tris, nfaces,
                                          nnodes, probe, inv_re, face_force, node_force, skipped);
}

template <typename T> void preload_ib() {
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_ib_force<T>);
    cudaFuncGetAttributes(&fa, k_ib_loads<T>);
}

#define FSEI_INST(T)                                                                           \
    template void launch_ib_force<T>(const GridDev &, const T *, const T *, const T *,        \
                                     const double *, const double *, const double *, int,     \
                                     double, T *, T *, T *, double *, int *, cudaStream_t);   \
    template void launch_ib_loads<T>(const GridDev &, const T *, const T *, const T *,        \
                                     const T *, const double *, const double *,               \
                                     const double *, const int *, const int *, int, int,      \
                                     double, double, double *, double *, int *,               \
                                     cudaStream_t);                                           \
    template void preload_ib<T>();
FSEI_INST(float)
FSEI_INST(double)
#undef FSEI_INST

}  // namespace fsei
