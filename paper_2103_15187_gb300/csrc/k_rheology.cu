// Carreau-Yasuda (shear-thinning) blood rheology (Sec. 2.1): the explicit
// remainder div(2 Re^-1 (eta(gdot) - 1) E) of the viscous stress beside the
// implicit Newtonian term, added to the advection term H of the step.
//
//   k_nn_visc   nu' = (eta(gdot) - 1) / Re at every cell centre: the normal
//               strain rates of the cell and its shear rates averaged from
//               the four surrounding edges of each kind, gdot = sqrt(2 E:E),
//               eta = eta_inf + (1 - eta_inf) (1 + (lam gdot)^a)^((n - 1)/a)
//   k_nn_div    div(2 nu' E) at the u, v, w points of every cell: normal
//               stresses at the centres, shear stresses at the edges with nu'
//               averaged over the cells around the edge (the two fluid cells
//               at a wall edge); z differences over dz_k (u, v) and hc_k (w);
//               0 on the bottom wall face
//
// Strain rates: E_xx = (u_{i+1} - u_i) / dx at the centres; E_xy = ((u_j -
// u_{j-1}) / dy + (v_i - v_{i-1}) / dx) / 2 at (x_i, y_j, zc_k); E_xz =
// ((u_k - u_{k-1}) / hc_k + (w_i - w_{i-1}) / dx) / 2 at (x_i, y_{j+1/2},
// z_k), E_yz alike; with walls a tangential velocity is 0 on the wall, half
// a cell below the first centre, and w = 0 on both wall faces.  One thread
// per cell, in the field precision.
#include "kernels.cuh"

namespace fsei {

namespace {

// neighbour access: periodic x, y; z periodic or walled (0 beyond a wall)
template <typename T> struct Nbr {
    const GridDev &g;
    FSEI_D int wx(int i) const { return i < 0 ? i + g.nx : (i >= g.nx ? i - g.nx : i); }
    FSEI_D int wy(int j) const { return j < 0 ? j + g.ny : (j >= g.ny ? j - g.ny : j); }
    // value of a centre-z field (u, v, nu) at cell (i, j, k)
    FSEI_D T c(const T *f, int i, int j, int k) const {
        if (g.walls && (k < 0 || k >= g.nz)) return T(0);
        const int kk = k < 0 ? k + g.nz : (k >= g.nz ? k - g.nz : k);
        return f[((size_t)kk * g.ny + wy(j)) * g.nx + wx(i)];
    }
    // w at face k (0 on both wall faces)
    FSEI_D T w(const T *f, int i, int j, int k) const {
        if (g.walls && (k <= 0 || k >= g.nz)) return T(0);
        const int kk = k < 0 ? k + g.nz : (k >= g.nz ? k - g.nz : k);
        return f[((size_t)kk * g.ny + wy(j)) * g.nx + wx(i)];
    }
    FSEI_D T ihc(int k) const { return Metric<T>::ihc(g)[k]; }   // k in [0, nz]
    FSEI_D T idz(int k) const {
        const int kk = k < 0 ? k + g.nz : (k >= g.nz ? k - g.nz : k);
        return Metric<T>::idz(g)[kk];
    }
};

template <typename T> struct Strain {
    const Nbr<T> &N;
    const T *u, *v, *w;
    T idx, idy;
    FSEI_D T exx(int i, int j, int k) const { return (N.c(u, i + 1, j, k) - N.c(u, i, j, k)) * idx; }
    FSEI_D T eyy(int i, int j, int k) const { return (N.c(v, i, j + 1, k) - N.c(v, i, j, k)) * idy; }
    FSEI_D T ezz(int i, int j, int k) const {
        return (N.w(w, i, j, k + 1) - N.w(w, i, j, k)) * N.idz(k);
    }
    FSEI_D T exy(int i, int j, int k) const {
        return T(0.5) * ((N.c(u, i, j, k) - N.c(u, i, j - 1, k)) * idy +
                         (N.c(v, i, j, k) - N.c(v, i - 1, j, k)) * idx);
    }
    // k in [0, nz]: the edge on face z_k
    FSEI_D T exz(int i, int j, int k) const {
        return T(0.5) * ((N.c(u, i, j, k) - N.c(u, i, j, k - 1)) * N.ihc(k) +
                         (N.w(w, i, j, k) - N.w(w, i - 1, j, k)) * idx);
    }
    FSEI_D T eyz(int i, int j, int k) const {
        return T(0.5) * ((N.c(v, i, j, k) - N.c(v, i, j, k - 1)) * N.ihc(k) +
                         (N.w(w, i, j, k) - N.w(w, i, j - 1, k)) * idy);
    }
};

}  // namespace

template <typename T>
FSEI_D void k_nn_visc(GridDev g, const T *__restrict__ u, const T *__restrict__ v,
                      const T *__restrict__ w, T *__restrict__ nu, T inv_re, T lam, T n, T a,
                      T eta_inf) {
    const Nbr<T> N{g};
    const Strain<T> S{N, u, v, w, fpick<T>(g.idx, g.fidx), fpick<T>(g.idy, g.fidy)};
    const size_t cells = (size_t)g.nx * g.ny * g.nz;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < cells;
         c += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((size_t)g.nx * g.ny));
        const T a1 = S.exx(i, j, k), a2 = S.eyy(i, j, k), a3 = S.ezz(i, j, k);
        const T q = T(0.25);
        const T bxy = q * (S.exy(i, j, k) + S.exy(i + 1, j, k) + S.exy(i, j + 1, k) + S.exy(i + 1, j + 1, k));
        const T bxz = q * (S.exz(i, j, k) + S.exz(i, j, k + 1) + S.exz(i + 1, j, k) + S.exz(i + 1, j, k + 1));
        const T byz = q * (S.eyz(i, j, k) + S.eyz(i, j, k + 1) + S.eyz(i, j + 1, k) + S.eyz(i, j + 1, k + 1));
        const T ee = a1 * a1 + a2 * a2 + a3 * a3 + T(2) * (bxy * bxy + bxz * bxz + byz * byz);
        const T gdot = sqrt(T(2) * ee);
        const T eta = eta_inf + (T(1) - eta_inf) * pow(T(1) + pow(lam * gdot, a), (n - T(1)) / a);
        nu[c] = (eta - T(1)) * inv_re;
    }
}

template <typename T>
FSEI_D void k_nn_div(GridDev g, const T *__restrict__ u, const T *__restrict__ v,
                     const T *__restrict__ w, const T *__restrict__ nu, T *__restrict__ hx,
                     T *__restrict__ hy, T *__restrict__ hz) {
    const Nbr<T> N{g};
    const Strain<T> S{N, u, v, w, fpick<T>(g.idx, g.fidx), fpick<T>(g.idy, g.fidy)};
    const T idx = S.idx, idy = S.idy, two = T(2), h = T(0.5), q = T(0.25);
    const int nz = g.nz;
    // nu' at the edges: xy (x_i, y_j, zc_k); xz (x_i, y_{j+1/2}, z_k); yz
    auto nxy = [&](int i, int j, int k) {
        return q * (N.c(nu, i, j, k) + N.c(nu, i - 1, j, k) + N.c(nu, i, j - 1, k) +
                    N.c(nu, i - 1, j - 1, k));
    };
    auto nxz = [&](int i, int j, int k) {
        if (g.walls && k == 0) return h * (N.c(nu, i, j, 0) + N.c(nu, i - 1, j, 0));
        if (g.walls && k == nz) return h * (N.c(nu, i, j, nz - 1) + N.c(nu, i - 1, j, nz - 1));
        return q * (N.c(nu, i, j, k) + N.c(nu, i - 1, j, k) + N.c(nu, i, j, k - 1) +
                    N.c(nu, i - 1, j, k - 1));
    };
    auto nyz = [&](int i, int j, int k) {
        if (g.walls && k == 0) return h * (N.c(nu, i, j, 0) + N.c(nu, i, j - 1, 0));
        if (g.walls && k == nz) return h * (N.c(nu, i, j, nz - 1) + N.c(nu, i, j - 1, nz - 1));
        return q * (N.c(nu, i, j, k) + N.c(nu, i, j - 1, k) + N.c(nu, i, j, k - 1) +
                    N.c(nu, i, j - 1, k - 1));
    };
    const size_t cells = (size_t)g.nx * g.ny * nz;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < cells;
         c += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((size_t)g.nx * g.ny));
        const T idzk = N.idz(k);
        // u point (x_i, y_{j+1/2}, zc_k)
        const T txx_r = two * N.c(nu, i, j, k) * S.exx(i, j, k);
        const T txx_l = two * N.c(nu, i - 1, j, k) * S.exx(i - 1, j, k);
        const T txy_u = two * nxy(i, j + 1, k) * S.exy(i, j + 1, k);
        const T txy_d = two * nxy(i, j, k) * S.exy(i, j, k);
        const T txz_u = two * nxz(i, j, k + 1) * S.exz(i, j, k + 1);
        const T txz_d = two * nxz(i, j, k) * S.exz(i, j, k);
        hx[c] = (txx_r - txx_l) * idx + (txy_u - txy_d) * idy + (txz_u - txz_d) * idzk;
        // v point (x_{i+1/2}, y_j, zc_k)
        const T tyy_u = two * N.c(nu, i, j, k) * S.eyy(i, j, k);
        const T tyy_d = two * N.c(nu, i, j - 1, k) * S.eyy(i, j - 1, k);
        const T txy_r = two * nxy(i + 1, j, k) * S.exy(i + 1, j, k);
        const T tyz_u = two * nyz(i, j, k + 1) * S.eyz(i, j, k + 1);
        const T tyz_d = two * nyz(i, j, k) * S.eyz(i, j, k);
        hy[c] = (txy_r - txy_d) * idx + (tyy_u - tyy_d) * idy + (tyz_u - tyz_d) * idzk;
        // w point (x_{i+1/2}, y_{j+1/2}, z_k); 0 on the bottom wall face
        if (g.walls && k == 0) {
            hz[c] = T(0);
        } else {
            const T txz_r = two * nxz(i + 1, j, k) * S.exz(i + 1, j, k);
            const T tyz_r = two * nyz(i, j + 1, k) * S.eyz(i, j + 1, k);
            const T tzz_u = two * N.c(nu, i, j, k) * S.ezz(i, j, k);
            const T tzz_d = two * N.c(nu, i, j, k - 1) * S.ezz(i, j, k - 1);
            hz[c] = (txz_r - txz_d) * idx + (tyz_r - tyz_d) * idy + (tzz_u - tzz_d) * N.ihc(k);
        }
    }
}

template <typename T> constexpr Kernel<k_nn_visc<T>, 256, 0> K_nn_visc{};
template <typename T> constexpr Kernel<k_nn_div<T>, 256, 0> K_nn_div{};

template <typename T>
void launch_non_newtonian(const GridDev &g, const T *u, const T *v, const T *w, Work<T> &W,
                          double re, const double cy[4], cudaStream_t st) {
    const size_t cells = (size_t)g.nx * g.ny * g.nz;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t want = (cells + 255) / 256;
    const int blocks = (int)(want < (size_t)sms * 8 ? want : (size_t)sms * 8);
    K_nn_visc<T>.launch(false, dim3(blocks), dim3(256), 0, st, g, u, v, w, W.nuc, T(1.0 / re),
                        T(cy[0]), T(cy[1]), T(cy[2]), T(cy[3]));
    K_nn_div<T>.launch(false, dim3(blocks), dim3(256), 0, st, g, u, v, w, (const T *)W.nuc,
                       W.nn0, W.nn1, W.nn2);
}

template <typename T> void preload_rheology() {
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, K_nn_visc<T>.solo());
    cudaFuncGetAttributes(&fa, K_nn_div<T>.solo());
}

#define FSEI_INST(T)                                                                           \
    template void launch_non_newtonian<T>(const GridDev &, const T *, const T *, const T *,    \
                                          Work<T> &, double, const double *, cudaStream_t);    \
    template void preload_rheology<T>();
FSEI_INST(float)
FSEI_INST(double)
#undef FSEI_INST

}  // namespace fsei
