// Reverse-time (adjoint) step of the literal Strang form on a periodic ring
// (internal header). One thread per cell; a step's adjoint reads only the
// adjoints after the step and the forward state before it, so no block-level
// synchronisation is needed and one launch handles one step.
//
// Forward step (periodic, sigma general):
//   H'_i = H_i + ch (E_{i+1} - E_i)
//   d'   = d + (Dl d + b);  z = T^T d';  d'' = d' + T (R(phi) - I) z,  phi_k = theta_k dt E_i
//   dn   = d'' + (Dl d'' + b);  p = w . dn + c
//   E'_i = ca E_i + cb ((H'_i - H'_{i-1}) / dx - p_i);  source at source_cell
// Objective J = dt sum_n (E^{n+1}_probe)^2: the reverse of step n adds
// 2 dt E^{n+1}_probe to the adjoint of E^{n+1}_probe.
#pragma once

#include "kernels.cuh"

namespace mln {

template <int N, typename R>
struct AdjConsts {
    R Dl[Dims<N>::D * Dims<N>::D];
    R T[Dims<N>::D * Dims<N>::D];
    R b[Dims<N>::D];
    R w[Dims<N>::D];
    R psi_dt[N - 1];
    R theta_dt[Dims<N>::Q];
};

template <typename R>
struct AdjArgs {
    const R *E0, *E1, *S0;        // forward E^n, E^{n+1} (cells), state d^{n-1/2} (SoA)
    const R *Ea, *Ha, *Sa;        // adjoints after the step (of E^{n+1}, H^{n+1/2}, d^{n+1/2})
    R *Eb, *Hb, *Sb;              // adjoints before the step (of E^n, H^{n-1/2}, d^{n-1/2})
    double *dsrc;                 // adjoint of this step's source sample (one double), or nullptr
    double *acc;                  // per-cell accumulators: entry k of cell i at k * n_cells + i (AccLayout)
    int64_t n_cells, mb, me, stride, source_cell, probe_cell;
    int32_t source_kind, pad_;
    double dt, E_step;            // dt; unused
    R ch, ca, cb, inv_dx;
};

// Accumulator layout (FP64): Dl_bar (D x D) | b_bar (D) | w_bar (D) | c_bar |
// T_bar (D x D) | theta_bar (q) | J
template <int N>
struct AccLayout {
    static constexpr int D = Dims<N>::D, Q = Dims<N>::Q;
    static constexpr int Dl = 0, b = D * D, w = b + D, c = w + D, T = c + 1, th = T + D * D, J = th + Q,
                         size = J + 1;
};

// Each cell owns one column of the accumulators and adds to it at every
// step (no atomics, no shuffles); mln_adjoint_reduce sums over the cells.
__device__ __forceinline__ void acc_add(double *acc, int64_t n, int64_t i, int idx, double v) {
    acc[idx * n + i] += v;
}

// acc_out[k] = sum_i acc[k * n + i], one block per k, fixed summation order.
__global__ void __launch_bounds__(256) mln_adjoint_reduce(const double *__restrict__ acc, int64_t n,
                                                          double *__restrict__ out) {
    __shared__ double part[256];
    const int k = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += acc[k * n + i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = part[0];
}

template <int N, typename R>
__global__ void __launch_bounds__(256) mln_adjoint_step(const __grid_constant__ AdjArgs<R> a,
                                                        const __grid_constant__ AdjConsts<N, R> k) {
    constexpr int D = Dims<N>::D, Q = Dims<N>::Q;
    using L = AccLayout<N>;
    const int64_t n = a.n_cells;
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    const bool live = i < n;
    const int64_t ii = live ? i : 0;
    const int64_t ip = ii + 1 == n ? 0 : ii + 1, im = ii == 0 ? n - 1 : ii - 1;
    const R jdt = static_cast<R>(2.0 * a.dt);

    // adjoint of E' at a cell, with the objective term and a hard source (which cuts the path)
    auto ebar_out = [&](int64_t c) -> R {
        R v = a.Ea[c];
        if (c == a.probe_cell) v += jdt * a.E1[c];
        if (a.dsrc != nullptr && a.source_kind == 1 && c == a.source_cell) v = R(0);
        return v;
    };
    R ep_i = R(0), ep_p = R(0), ep_m = R(0);
    if (live) {
        ep_i = ebar_out(ii);
        ep_p = ebar_out(ip);
        ep_m = ebar_out(im);
    }
    // source sample: soft adds it, hard sets E' to it; both pass the adjoint of E'
    if (live && a.dsrc != nullptr && ii == a.source_cell) {
        R v = a.Ea[ii];
        if (ii == a.probe_cell) v += jdt * a.E1[ii];
        *a.dsrc = static_cast<double>(v);
    }
    if (live && ii == a.probe_cell) {
        const double e1 = static_cast<double>(a.E1[ii]);
        a.acc[L::J * n + ii] += a.dt * e1 * e1;
    }
    // adjoint of H'_i and H'_{i-1} (used by E'_i, E'_{i+1} and E'_{i-1}, E'_i)
    R hh_i = R(0), hh_m = R(0);
    if (live) {
        hh_i = a.Ha[ii] + a.cb * a.inv_dx * (ep_i - ep_p);
        hh_m = a.Ha[im] + a.cb * a.inv_dx * (ep_m - ep_i);
        a.Hb[ii] = hh_i;
    }
    R eb = live ? a.ca * ep_i + a.ch * (hh_m - hh_i) : R(0);

    const bool medium = live && ii >= a.mb && ii < a.me;
    const int64_t m = ii - a.mb;
    // forward recompute of the cell (zeros for lanes outside the medium)
    R d[D], y[D], z[D], y2[D], dn[D], sn[Q], c1[Q];
    const R e = live ? a.E0[ii] : R(0);
#pragma unroll
    for (int j = 0; j < D; ++j) d[j] = medium ? a.S0[j * a.stride + m] : R(0);
    affine_inc<D>(y, k.Dl, d, k.b);
    matTvec<D>(z, k.T, y);
    plane_terms<N>(k.psi_dt, e, sn, c1);
    R dz[D];
#pragma unroll
    for (int j = 0; j < D; ++j) dz[j] = R(0);
#pragma unroll
    for (int p = 0; p < Q; ++p) {
        dz[2 * p] = fma(c1[p], z[2 * p], sn[p] * z[2 * p + 1]);
        dz[2 * p + 1] = fma(c1[p], z[2 * p + 1], -(sn[p] * z[2 * p]));
    }
#pragma unroll
    for (int j = 0; j < D; ++j) y2[j] = y[j];
    matvec_acc<D>(y2, k.T, dz);
    affine_inc<D>(dn, k.Dl, y2, k.b);
    if (!medium) {
#pragma unroll
        for (int j = 0; j < D; ++j) d[j] = y[j] = z[j] = y2[j] = dn[j] = dz[j] = R(0);
    }

    // reverse: p = w . dn + c with pbar = -cb * Ebar'_i
    const R pbar = medium ? -a.cb * ep_i : R(0);
    R dnb[D];
#pragma unroll
    for (int j = 0; j < D; ++j) dnb[j] = (medium ? a.Sa[j * a.stride + m] : R(0)) + pbar * k.w[j];
    // dn = A0 y2 + b
    R y2b[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        R acc = dnb[j];
#pragma unroll
        for (int l = 0; l < D; ++l) acc = fma(k.Dl[l * D + j], dnb[l], acc);
        y2b[j] = acc;
    }
    // y2 = y + T (R - I) T^T y: zb = T^T y2b; ybar = y2b + T (R^T - I) zb
    R zb[D], dzb[D];
    matTvec<D>(zb, k.T, y2b);
#pragma unroll
    for (int j = 0; j < D; ++j) dzb[j] = R(0);
    R e_term = R(0);
    double thb[Q];
#pragma unroll
    for (int p = 0; p < Q; ++p) {
        const R zx = z[2 * p], zy = z[2 * p + 1], bx = zb[2 * p], by = zb[2 * p + 1];
        dzb[2 * p] = fma(c1[p], bx, -(sn[p] * by));
        dzb[2 * p + 1] = fma(c1[p], by, sn[p] * bx);
        const R cs = R(1) + c1[p];
        // d/dphi of R z = (-s zx + c zy, -c zx - s zy)
        const R br = bx * fma(-sn[p], zx, cs * zy) + by * fma(-cs, zx, -(sn[p] * zy));
        e_term = fma(k.theta_dt[p], br, e_term);
        thb[p] = static_cast<double>(br) * static_cast<double>(e) * a.dt;
    }
    R yb[D];
#pragma unroll
    for (int j = 0; j < D; ++j) yb[j] = y2b[j];
    matvec_acc<D>(yb, k.T, dzb);
    // y = A0 d + b
    R db[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        R acc = yb[j];
#pragma unroll
        for (int l = 0; l < D; ++l) acc = fma(k.Dl[l * D + j], yb[l], acc);
        db[j] = acc;
    }
    if (medium) {
#pragma unroll
        for (int j = 0; j < D; ++j) a.Sb[j * a.stride + m] = db[j];
        eb += e_term;
    }
    if (live) a.Eb[ii] = eb;

    // parameter accumulators of this cell
    if (!medium) return;
#pragma unroll
    for (int r = 0; r < D; ++r) {
#pragma unroll
        for (int c = 0; c < D; ++c)
            acc_add(a.acc, n, ii, L::Dl + r * D + c,
                    static_cast<double>(dnb[r]) * y2[c] + static_cast<double>(yb[r]) * d[c]);
        acc_add(a.acc, n, ii, L::b + r, static_cast<double>(dnb[r]) + yb[r]);
        acc_add(a.acc, n, ii, L::w + r, static_cast<double>(pbar) * dn[r]);
        // T_bar = y2b (dz)^T + y (dzb)^T on the plane columns
#pragma unroll
        for (int c = 0; c < 2 * Q; ++c)
            acc_add(a.acc, n, ii, L::T + r * D + c,
                    static_cast<double>(y2b[r]) * dz[c] + static_cast<double>(y[r]) * dzb[c]);
    }
    acc_add(a.acc, n, ii, L::c, static_cast<double>(pbar));
#pragma unroll
    for (int p = 0; p < Q; ++p) acc_add(a.acc, n, ii, L::th + p, thb[p]);
}

}  // namespace mln
