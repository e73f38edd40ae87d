// Reverse-time (adjoint) step of the literal Strang form, on a periodic ring
// or an open grid (held cell 0 with a hard or soft source, first-order Mur at
// the right end) (internal header). A step's adjoint reads only the adjoints
// after the step and the forward state before it, so no block-level
// synchronisation is needed and one launch handles one step.
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
    int32_t source_kind, boundary;  // boundary: 0 ring, 1 open (held cell 0, Mur at n - 1)
    double dt, E_step;            // dt; unused
    R ch, ca, cb, inv_dx, kappa;
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

// Lanes per cell of the row-parallel reverse step: a power of two >= D.
template <int N>
struct AdjLanes {
    static constexpr int D = Dims<N>::D;
    static constexpr int value = D <= 4 ? 4 : (D <= 8 ? 8 : 16);
};

// The reverse step with one lane per component: the AdjLanes lanes of a cell
// each own one row r < D of every vector and of every product, and read the
// other components of a product's input by shuffles within the cell's lanes.
// Each component gets the operations, in the order, that one thread per cell
// would apply to it (sums over an index run in ascending order), so the lane
// split changes no bits; small rings keep all SMs busy and each lane's
// dependency chains are D times shorter.
//
// Forward step being differentiated (sigma general):
//   H'_i = H_i + ch (E_{i+1} - E_i)                     i in the H range
//   d'   = d + (Dl d + b);  z = T^T d';  d'' = d' + T (R(phi) - I) z,  phi_k = theta_k dt E_i
//   dn   = d'' + (Dl d'' + b);  p = w . dn + c
//   E'_i = ca E_i + cb ((H'_i - H'_{i-1}) / dx - p_i)   i in the E range
//   open grid: E'_0 = E_0 (held); E'_{n-1} = E_{n-2} + kappa (E'_{n-2} - E_{n-1}) (Mur,
//   from E'_{n-2} before any source); then the source at source_cell (hard:
//   replace, soft: add). Ring: every cell in both ranges, indices modulo n;
//   open grid: H range 0..n-2, E range 1..n-2.
// Objective J = dt sum_n (E^{n+1}_probe)^2: the reverse of step n adds
// 2 dt E^{n+1}_probe to the adjoint of E^{n+1}_probe.
//
// Reverse of the field part, per cell i, with Ebar' the adjoint of E^{n+1}:
//   m      = adjoint of the Mur cell's new value (0 under a hard source there)
//   epre_i = adjoint of cell i's E update before source and Mur: Ebar'_i (0
//            under a hard source at i), plus kappa m at i = n - 2; 0 outside the E range
//   Hbar_i = Hbar'_i + cb/dx (epre_i - epre_{i+1})           i in the H range
//   Ebar_i = ca epre_i + ch (Hbar_{i-1} - Hbar_i)  (terms in the H range only)
//            + Ebar'_0 at the held cell 0 (not under a hard source),
//            + m at n - 2, - kappa m at n - 1, + the medium's term
//   pbar_i = -cb epre_i
template <int N, typename R>
__global__ void __launch_bounds__(128) mln_adjoint_step_rows(const __grid_constant__ AdjArgs<R> a,
                                                             const __grid_constant__ AdjConsts<N, R> k) {
    constexpr int D = Dims<N>::D, Q = Dims<N>::Q, LN = AdjLanes<N>::value;
    using L = AccLayout<N>;
    const int64_t n = a.n_cells;
    const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    const int64_t i = t / LN;
    const int r = static_cast<int>(t % LN);
    const bool live = i < n;
    const bool row = live && r < D;
    const int64_t ii = live ? i : 0;
    const bool periodic = a.boundary == 0;
    const int64_t ip = ii + 1 == n ? 0 : ii + 1, im = ii == 0 ? n - 1 : ii - 1;
    const R jdt = static_cast<R>(2.0 * a.dt);
    const unsigned full = 0xffffffffu;
    auto get = [&](R v, int src) { return __shfl_sync(full, v, src, LN); };  // component src of this cell
    const int rr = r < D ? r : 0;
    // this lane's rows and columns of the constant matrices
    R dl_row[D], dl_col[D], t_row[D], t_col[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        dl_row[j] = k.Dl[rr * D + j];
        dl_col[j] = k.Dl[j * D + rr];
        t_row[j] = k.T[rr * D + j];
        t_col[j] = k.T[j * D + rr];
    }
    const R b_r = k.b[rr], w_r = k.w[rr];

    // scalars of the cell (every lane; lane 0 writes)
    auto ebar_new = [&](int64_t c) -> R {  // adjoint of E^{n+1}_c, with the objective's term
        R v = a.Ea[c];
        if (c == a.probe_cell) v += jdt * a.E1[c];
        return v;
    };
    auto hard = [&](int64_t c) { return a.dsrc != nullptr && a.source_kind == 1 && c == a.source_cell; };
    const R mbar = (!periodic && live && !hard(n - 1)) ? ebar_new(n - 1) : R(0);
    auto epre = [&](int64_t c) -> R {
        if (!periodic && (c <= 0 || c >= n - 1)) return R(0);
        R v = hard(c) ? R(0) : ebar_new(c);
        if (!periodic && c == n - 2) v += a.kappa * mbar;
        return v;
    };
    auto in_h = [&](int64_t c) { return periodic || c <= n - 2; };
    R ep_i = R(0), ep_p = R(0), ep_m = R(0);
    if (live) {
        ep_i = epre(ii);
        if (periodic || ii + 1 < n) ep_p = epre(ip);
        if (periodic || ii >= 1) ep_m = epre(im);
    }
    if (live && r == 0 && a.dsrc != nullptr && ii == a.source_cell) {
        R v = a.Ea[ii];
        if (ii == a.probe_cell) v += jdt * a.E1[ii];
        *a.dsrc = static_cast<double>(v);
    }
    if (live && r == 0 && ii == a.probe_cell) {
        const double e1 = static_cast<double>(a.E1[ii]);
        a.acc[L::J * n + ii] += a.dt * e1 * e1;
    }
    R hh_i = R(0), hh_m = R(0);
    const bool has_m = periodic || ii >= 1;  // H_{i-1/2} exists
    if (live) {
        hh_i = a.Ha[ii] + (in_h(ii) ? a.cb * a.inv_dx * (ep_i - ep_p) : R(0));
        if (has_m) hh_m = a.Ha[im] + (in_h(im) ? a.cb * a.inv_dx * (ep_m - ep_i) : R(0));
        if (r == 0) a.Hb[ii] = hh_i;
    }
    R eb = live ? a.ca * ep_i + a.ch * ((has_m ? hh_m : R(0)) - (in_h(ii) ? hh_i : R(0))) : R(0);
    if (live && !periodic) {
        if (ii == 0 && !hard(0)) eb += ebar_new(0);  // held: E^{n+1}_0 = E^n_0
        if (ii == n - 2) eb += mbar;                 // E^n_{n-2} in the Mur rule
        if (ii == n - 1) eb -= a.kappa * mbar;       // E^n_{n-1} in the Mur rule
    }

    const bool medium = live && ii >= a.mb && ii < a.me;
    const bool mrow = medium && r < D;
    const int64_t m = ii - a.mb;
    const R e = live ? a.E0[ii] : R(0);
    // forward recompute of the cell, one component per lane
    const R d = mrow ? a.S0[r * a.stride + m] : R(0);
    R y;  // y = d + (Dl d + b)
    {
        R acc = b_r;
#pragma unroll
        for (int j = 0; j < D; ++j) acc = fma(dl_row[j], get(d, j), acc);
        y = d + acc;
    }
    R z;  // z = T^T y
    {
        R acc = t_col[0] * get(y, 0);
#pragma unroll
        for (int j = 1; j < D; ++j) acc = fma(t_col[j], get(y, j), acc);
        z = acc;
    }
    R sn[Q], c1[Q];
    plane_terms<N>(k.psi_dt, e, sn, c1);
    const int pl = rr / 2;
    const R z_pair = __shfl_xor_sync(full, z, 1, LN);
    R dz = R(0);
    if (r < 2 * Q) dz = (r % 2 == 0) ? fma(c1[pl], z, sn[pl] * z_pair) : fma(c1[pl], z, -(sn[pl] * z_pair));
    R y2;  // y2 = y + T dz
    {
        R acc = t_row[0] * get(dz, 0);
#pragma unroll
        for (int j = 1; j < D; ++j) acc = fma(t_row[j], get(dz, j), acc);
        y2 = y + acc;
    }
    R dn;  // dn = y2 + (Dl y2 + b)
    {
        R acc = b_r;
#pragma unroll
        for (int j = 0; j < D; ++j) acc = fma(dl_row[j], get(y2, j), acc);
        dn = y2 + acc;
    }
    R dv = d, yv = y, zv = z, y2v = y2, dnv = dn, dzv = dz;
    if (!mrow) dv = yv = zv = y2v = dnv = dzv = R(0);

    // reverse
    const R pbar = medium ? -a.cb * ep_i : R(0);
    const R dnb = (mrow ? a.Sa[r * a.stride + m] : R(0)) + pbar * w_r;
    R y2b;  // y2b = dnb + Dl^T dnb
    {
        R acc = dnb;
#pragma unroll
        for (int l = 0; l < D; ++l) acc = fma(dl_col[l], get(dnb, l), acc);
        y2b = acc;
    }
    R zb;  // zb = T^T y2b
    {
        R acc = t_col[0] * get(y2b, 0);
#pragma unroll
        for (int j = 1; j < D; ++j) acc = fma(t_col[j], get(y2b, j), acc);
        zb = acc;
    }
    const R zb_pair = __shfl_xor_sync(full, zb, 1, LN);
    const R zv_pair = __shfl_xor_sync(full, zv, 1, LN);
    R dzb = R(0), br = R(0);
    if (r < 2 * Q) {
        const bool even = r % 2 == 0;
        dzb = even ? fma(c1[pl], zb, -(sn[pl] * zb_pair)) : fma(c1[pl], zb, sn[pl] * zb_pair);
        if (even) {
            const R zx = zv, zy = zv_pair, bx = zb, by = zb_pair, cs = R(1) + c1[pl];
            br = bx * fma(-sn[pl], zx, cs * zy) + by * fma(-cs, zx, -(sn[pl] * zy));
        }
    }
    R e_term = R(0);
#pragma unroll
    for (int p = 0; p < Q; ++p) e_term = fma(k.theta_dt[p], get(br, 2 * p), e_term);
    R yb;  // yb = y2b + T dzb
    {
        R acc = t_row[0] * get(dzb, 0);
#pragma unroll
        for (int j = 1; j < D; ++j) acc = fma(t_row[j], get(dzb, j), acc);
        yb = y2b + acc;
    }
    R db;  // db = yb + Dl^T yb
    {
        R acc = yb;
#pragma unroll
        for (int l = 0; l < D; ++l) acc = fma(dl_col[l], get(yb, l), acc);
        db = acc;
    }
    if (mrow) a.Sb[r * a.stride + m] = db;
    if (medium) eb += e_term;
    if (live && r == 0) a.Eb[ii] = eb;

    // parameter accumulators of this cell: lane r owns row r (shuffles for all lanes)
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const R y2c = get(y2v, c), dc = get(dv, c);
        if (mrow) acc_add(a.acc, n, ii, L::Dl + r * D + c, static_cast<double>(dnb) * y2c + static_cast<double>(yb) * dc);
    }
    if (mrow) {
        acc_add(a.acc, n, ii, L::b + r, static_cast<double>(dnb) + yb);
        acc_add(a.acc, n, ii, L::w + r, static_cast<double>(pbar) * dnv);
    }
#pragma unroll
    for (int c = 0; c < 2 * Q; ++c) {
        const R dzc = get(dzv, c), dzbc = get(dzb, c);
        if (mrow)
            acc_add(a.acc, n, ii, L::T + r * D + c, static_cast<double>(y2b) * dzc + static_cast<double>(yv) * dzbc);
    }
    if (medium && r == 0) acc_add(a.acc, n, ii, L::c, static_cast<double>(pbar));
    if (medium && r < 2 * Q && r % 2 == 0)
        acc_add(a.acc, n, ii, L::th + r / 2, static_cast<double>(br) * static_cast<double>(e) * a.dt);
}

}  // namespace mln
