// Fused Maxwell + Liouville step kernels for sm_103a (internal header).
//
// One thread owns one grid cell. A thread block owns a tile of cells and
// advances it by up to `halo` time steps per launch (temporal blocking):
// it loads the tile plus `halo` cells on each side, keeps E_z and H_y of the
// loaded span in shared memory and each medium cell's adjoint vector in
// registers, and after `nsteps <= halo` steps writes back only the tile,
// whose values depend on nothing outside the loaded span (a step moves
// information by one cell). Cells near the span's edges compute throw-away
// values; the cost is 2*halo/tile extra cell updates.
//
// Per step (Fig. 1 and Eq. 23 of Riesch & Jirauschek):
//   H^{n+1/2}_{i+1/2} = H^{n-1/2}_{i+1/2} + dt/(mu dx) (E^n_{i+1} - E^n_i)     (Eq. 1b)
//   medium cells: d^{n-1/2} -> d^{n+1/2} with E^n_i                          (Eq. 23a-c)
//                 dP/dt^{n+1/2}_i = w . d^{n+1/2} + c                        (Eq. 17)
//   E^{n+1}_i = ca E^n_i + cb ((H_{i+1/2} - H_{i-1/2})/dx - dP/dt_i)          (Eq. 1a)
//   boundary (ring, or held cell 0 + first-order Mur at the right), source.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mln {

template <int N>
struct Dims {
    static constexpr int D = N * N - 1;      // adjoint dimension
    static constexpr int Q = N * (N - 1) / 2; // rotation planes of U
};

// Constants of the literal Strang form (Eq. 23 with the diagonalisation of Eq. 25):
// d' = A0 d + b; z = T^T d'; z rotated plane by plane by theta_dt[k] * E;
// d'' = T z; d_new = A0 d'' + b; dP/dt = w . d_new + c.
template <int N, typename R>
struct StrangConsts {
    R A0[Dims<N>::D * Dims<N>::D];
    R T[Dims<N>::D * Dims<N>::D];
    R b[Dims<N>::D];
    R w[Dims<N>::D];
    R theta_dt[Dims<N>::Q];
    R c;
};

// Constants of the rotated form: state p = T^T (A0 d + b);
// z = R(E) p; dP/dt = wr . z + cr; p_new = C z + cp.
template <int N, typename R>
struct RotConsts {
    R C[Dims<N>::D * Dims<N>::D];
    R cp[Dims<N>::D];
    R wr[Dims<N>::D];
    R theta_dt[Dims<N>::Q];
    R cr;
};

template <typename R>
struct BlockArgs {
    const R *E_in;
    const R *H_in;
    const R *s_in;
    R *E_out;
    R *H_out;
    R *s_out;
    const double *src;     // samples of this launch's steps, or nullptr
    unsigned int *flags;   // bit 0: non-finite E seen
    int64_t n_cells, mb, me, stride, source_cell;
    int32_t nsteps, halo, tile, boundary, source_kind, pad_;
    R ch, ca, cb, inv_dx, kappa;
};

__device__ __forceinline__ void sincos_r(double x, double *s, double *c) { sincos(x, s, c); }
__device__ __forceinline__ void sincos_r(float x, float *s, float *c) { sincosf(x, s, c); }

// Turn plane k = (z[2k], z[2k+1]) by phi_k = theta_dt[k] * e:
// (x, y) -> (x cos phi + y sin phi, -x sin phi + y cos phi), the flow of the
// block [[0, theta], [-theta, 0]] of T^T U T over E dt.
template <int N, typename R>
__device__ __forceinline__ void rotate_planes(R (&z)[Dims<N>::D], const R *theta_dt, R e) {
#pragma unroll
    for (int k = 0; k < Dims<N>::Q; ++k) {
        R sn, cs;
        sincos_r(theta_dt[k] * e, &sn, &cs);
        R x = z[2 * k], y = z[2 * k + 1];
        z[2 * k] = fma(cs, x, sn * y);
        z[2 * k + 1] = fma(cs, y, -(sn * x));
    }
}

// y = A x (+ b) with A row-major D x D held in the constant bank.
template <int D, typename R>
__device__ __forceinline__ void matvec(R (&y)[D], const R *A, const R (&x)[D]) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
        R acc = A[i * D] * x[0];
#pragma unroll
        for (int j = 1; j < D; ++j) acc = fma(A[i * D + j], x[j], acc);
        y[i] = acc;
    }
}

template <int D, typename R>
__device__ __forceinline__ void matvec_bias(R (&y)[D], const R *A, const R (&x)[D], const R *b) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
        R acc = b[i];
#pragma unroll
        for (int j = 0; j < D; ++j) acc = fma(A[i * D + j], x[j], acc);
        y[i] = acc;
    }
}

template <int D, typename R>
__device__ __forceinline__ void matTvec(R (&y)[D], const R *A, const R (&x)[D]) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
        R acc = A[k] * x[0];
#pragma unroll
        for (int i = 1; i < D; ++i) acc = fma(A[i * D + k], x[i], acc);
        y[k] = acc;
    }
}

template <int D, typename R>
__device__ __forceinline__ R dot_bias(const R *w, const R (&x)[D], R c) {
    R acc = c;
#pragma unroll
    for (int i = 0; i < D; ++i) acc = fma(w[i], x[i], acc);
    return acc;
}

// One Liouville step of one cell; returns dP/dt^{n+1/2}.
// Only two D-vectors are live at a time (s and y) to keep register pressure low.
template <int N, typename R>
__device__ __forceinline__ R cell_step(R (&s)[Dims<N>::D], R e, const StrangConsts<N, R> &k) {
    constexpr int D = Dims<N>::D;
    R y[D];
    matvec_bias<D>(y, k.A0, s, k.b);   // d' = A0 d + b           (Eq. 23a)
    matTvec<D>(s, k.T, y);             // into the eigenbasis of U
    rotate_planes<N>(s, k.theta_dt, e); // exp(Lambda E dt), real form (Eqs. 23b, 25)
    matvec<D>(y, k.T, s);              // d'' = T z
    matvec_bias<D>(s, k.A0, y, k.b);   // d = A0 d'' + b          (Eq. 23c)
    return dot_bias<D>(k.w, s, k.c);   // dP/dt = w . d + c       (Eq. 17)
}

template <int N, typename R>
__device__ __forceinline__ R cell_step(R (&s)[Dims<N>::D], R e, const RotConsts<N, R> &k) {
    constexpr int D = Dims<N>::D;
    R z[D];
#pragma unroll
    for (int i = 0; i < D; ++i) z[i] = s[i];
    rotate_planes<N>(z, k.theta_dt, e);
    R dpdt = dot_bias<D>(k.wr, z, k.cr);
    matvec_bias<D>(s, k.C, z, k.cp);
    return dpdt;
}

// Blocks have at most kMaxThreads threads, which leaves up to 128 registers per thread.
constexpr int kMaxThreads = 512;

template <int N, typename R, typename K>
__global__ void __launch_bounds__(kMaxThreads) mln_block_kernel(const __grid_constant__ BlockArgs<R> a,
                                                         const __grid_constant__ K k) {
    constexpr int D = Dims<N>::D;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sE = reinterpret_cast<R *>(smem_raw);
    R *sH = sE + blockDim.x;

    const int j = threadIdx.x;
    const int64_t n = a.n_cells;
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * a.tile;
    const int64_t t1 = min(t0 + a.tile, n);
    const int L = static_cast<int>(t1 - t0) + 2 * a.halo;
    const bool periodic = a.boundary == 0;
    const int64_t g = t0 - a.halo + j;
    int64_t gm = g;
    bool loaded = j < L;
    if (periodic) {
        gm = g % n;
        if (gm < 0) gm += n;
    } else {
        loaded = loaded && g >= 0 && g < n;
    }
    const bool medium = loaded && gm >= a.mb && gm < a.me;
    const int64_t m = gm - a.mb;

    R e = loaded ? a.E_in[gm] : R(0);
    R h = loaded ? a.H_in[gm] : R(0);
    sE[j] = e;
    sH[j] = h;
    R s[D];
#pragma unroll
    for (int i = 0; i < D; ++i) s[i] = medium ? a.s_in[i * a.stride + m] : R(0);

    // H_{i+1/2} exists for every cell of a ring and for cells 0..n-2 of an open grid;
    // it needs E of the next loaded cell.
    const bool h_upd = loaded && (j + 1 < L) && (periodic || gm < n - 1);
    // E needs H_{i-1/2} of the previous loaded cell. On an open grid cell 0 is held
    // (hard source only) and cell n-1 is set by the Mur rule of cell n-2's thread.
    const bool e_upd = loaded && j >= 1 && (periodic || (gm > 0 && gm < n - 1));
    const bool mur = !periodic && loaded && gm == n - 2 && j + 1 < L;
    const bool is_src = a.src != nullptr && loaded && gm == a.source_cell;
    __syncthreads();

    for (int st = 0; st < a.nsteps; ++st) {
        if (h_upd) {
            h = fma(a.ch, sE[j + 1] - e, h);
            sH[j] = h;
        }
        __syncthreads();
        R dpdt = R(0);
        if (medium) dpdt = cell_step<N>(s, e, k);
        R en = e;
        if (e_upd) en = fma(a.ca, e, a.cb * fma(h - sH[j - 1], a.inv_dx, -dpdt));
        R e_mur = R(0);
        if (mur) e_mur = fma(a.kappa, en - sE[j + 1], e);
        if (is_src) {
            R v = static_cast<R>(a.src[st]);
            en = (a.source_kind == 1) ? v : en + v;
        }
        if (mur) {
            if (a.src != nullptr && a.source_cell == n - 1) {
                R v = static_cast<R>(a.src[st]);
                e_mur = (a.source_kind == 1) ? v : e_mur + v;
            }
            sE[j + 1] = e_mur;
        }
        e = en;
        if (loaded && !(!periodic && gm == n - 1)) sE[j] = e;
        __syncthreads();
        // the Mur cell takes its new value from shared memory
        if (!periodic && loaded && gm == n - 1) e = sE[j];
    }

    const bool interior = loaded && j >= a.halo && j < a.halo + static_cast<int>(t1 - t0);
    if (interior) {
        a.E_out[gm] = e;
        a.H_out[gm] = h;
        if (medium) {
#pragma unroll
            for (int i = 0; i < D; ++i) a.s_out[i * a.stride + m] = s[i];
        }
        if (!isfinite(e)) atomicOr(a.flags, 1u);
    }
}

}  // namespace mln
