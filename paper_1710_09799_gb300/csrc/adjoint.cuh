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

// Arguments of the temporally blocked reverse sweep: one launch runs the
// reverse of steps j_hi, j_hi - 1, ..., j_hi - nsteps + 1 of a recomputed
// segment over tiles of `tile` cells with `halo` cells on the left and
// halo (+ 1 on an open grid: the Mur rule couples cell n - 3 to n - 1 in one
// step) on the right.
template <typename R>
struct AdjBlockArgs {
    const unsigned char *rec;  // recorded forward sets of the segment: set j at rec + j * rec_set
    int64_t rec_set, off_E;    // bytes per set; offset of E within a set (the state S at offset 0)
    int32_t j_hi, nsteps, halo, tile;
    const R *Ea, *Ha, *Sa;     // adjoints after step j_hi (of E^{n+1}, H^{n+1/2}, d^{n+1/2})
    R *Eb, *Hb, *Sb;           // adjoints before step j_hi - nsteps + 1
    double *dsrc;              // adjoint of the source sample of segment step j at dsrc[j], or nullptr
    double *acc;               // per-cell accumulators: entry k of cell i at k * n_cells + i (AccLayout)
    int64_t n_cells, mb, me, stride, source_cell, probe_cell;
    int32_t source_kind, boundary;  // boundary: 0 ring, 1 open (held cell 0, Mur at n - 1)
    double dt;
    R ch, ca, cb, inv_dx, kappa;
};

// The constant matrices as one lane needs them (its row r and column r of Dl
// and T): held in registers in FP32; in FP64, whose arithmetic is slow
// enough that shared-memory reads cost nothing, read from a padded copy in
// shared memory (rows of D + 1 entries: conflict-free for rows and columns),
// which leaves the registers to the accumulators.
template <int N, typename R, bool kRegs>
struct AdjLaneConsts;
template <int N, typename R>
struct AdjLaneConsts<N, R, true> {
    static constexpr int D = Dims<N>::D;
    R dlr[D], dlc[D], tr[D], tc[D];
    __device__ __forceinline__ void init(const AdjConsts<N, R> &k, int rr, R *) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            dlr[j] = k.Dl[rr * D + j];
            dlc[j] = k.Dl[j * D + rr];
            tr[j] = k.T[rr * D + j];
            tc[j] = k.T[j * D + rr];
        }
    }
    __device__ __forceinline__ R dl_row(int j) const { return dlr[j]; }
    __device__ __forceinline__ R dl_col(int j) const { return dlc[j]; }
    __device__ __forceinline__ R t_row(int j) const { return tr[j]; }
    __device__ __forceinline__ R t_col(int j) const { return tc[j]; }
};
template <int N, typename R>
struct AdjLaneConsts<N, R, false> {
    static constexpr int D = Dims<N>::D, P = D + 1;
    const R *dl, *t;  // shared memory, [D][D + 1] each
    int rr;
    // block-cooperative: copy Dl and T into the padded layout (needs a barrier after)
    __device__ __forceinline__ void init(const AdjConsts<N, R> &k, int r, R *sm) {
        for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
            sm[(e / D) * P + e % D] = k.Dl[e];
            sm[D * P + (e / D) * P + e % D] = k.T[e];
        }
        dl = sm;
        t = sm + D * P;
        rr = r;
    }
    __device__ __forceinline__ R dl_row(int j) const { return dl[rr * P + j]; }
    __device__ __forceinline__ R dl_col(int j) const { return dl[j * P + rr]; }
    __device__ __forceinline__ R t_row(int j) const { return t[rr * P + j]; }
    __device__ __forceinline__ R t_col(int j) const { return t[j * P + rr]; }
};

// Shared memory of the blocked reverse kernel: the padded constants (FP64)
// and two field arrays of the block's cells.
template <int N, typename R>
__host__ __device__ constexpr size_t adj_block_smem(int cells) {
    return (sizeof(R) == 8 ? 2 * Dims<N>::D * (Dims<N>::D + 1) * sizeof(R) : 0) + 2 * static_cast<size_t>(cells) * sizeof(R);
}

// The temporally blocked reverse sweep with one lane per component: the
// AdjLanes lanes of a cell each own one row r < D of every vector and of
// every product and read the other components of a product's input by
// shuffles within the cell's lanes; each lane also owns row r of the
// outer-product gradients, summed in registers over the launch's steps and
// added to the cell's accumulator column once at the end (interior cells
// only: halo cells are the neighbouring tiles' interior).
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
// Per step two barriers: after epre (read by the left neighbour) and after
// Hbar (read by the right neighbour). The cell n - 2 keeps the Mur cell's
// Ebar itself (the Mur cell is vacuum: Ebar_{n-1} = ch Hbar_{n-2} - kappa m),
// so reading it needs no third barrier.
template <int N, typename R>
__global__ void __launch_bounds__(512) mln_adjoint_block(const __grid_constant__ AdjBlockArgs<R> a,
                                                         const __grid_constant__ AdjConsts<N, R> k) {
    constexpr int D = Dims<N>::D, Q = Dims<N>::Q, LN = AdjLanes<N>::value;
    constexpr bool kRegs = sizeof(R) == 4;
    using L = AccLayout<N>;
    extern __shared__ __align__(16) unsigned char adj_smem[];
    R *smc = reinterpret_cast<R *>(adj_smem);
    const int cells = blockDim.x / LN;
    R *sEp = smc + (kRegs ? 0 : 2 * D * (D + 1));  // epre of each cell
    R *sHh = sEp + cells;                            // new Hbar of each cell

    const int64_t n = a.n_cells;
    const bool periodic = a.boundary == 0;
    const int lc = threadIdx.x / LN, r = threadIdx.x % LN, rr = r < D ? r : 0;
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * a.tile;
    const int64_t t1 = min(t0 + a.tile, n);
    const int lh = a.halo, rh = a.halo + (periodic ? 0 : 1);
    const int span = static_cast<int>(t1 - t0) + lh + rh;
    const int64_t g = t0 - lh + lc;
    bool loaded = lc < span;
    int64_t gm = g;
    if (periodic) gm = wrap_index(g, n);
    else loaded = loaded && g >= 0 && g < n;
    const int64_t ii = loaded ? gm : 0;
    const bool medium = loaded && ii >= a.mb && ii < a.me;
    const bool mrow = medium && r < D;
    const int64_t m = ii - a.mb;
    const bool interior = loaded && lc >= lh && lc < lh + static_cast<int>(t1 - t0);
    const bool in_h = loaded && (periodic || ii <= n - 2);
    const bool in_e = loaded && (periodic || (ii >= 1 && ii <= n - 2));
    const bool has_m = loaded && (periodic || ii >= 1) && lc >= 1;
    const bool has_p = loaded && (periodic || ii + 1 <= n - 1) && lc + 1 < span;
    const bool hard_src = a.dsrc != nullptr && a.source_kind == 1;
    const bool is_src = a.dsrc != nullptr && loaded && ii == a.source_cell;
    const bool is_probe = loaded && ii == a.probe_cell;
    const bool before_mur = !periodic && loaded && ii == n - 2;
    const R jdt = static_cast<R>(2.0 * a.dt), cbdx = a.cb * a.inv_dx;
    const unsigned full = 0xffffffffu;
    auto get = [&](R v, int src) { return __shfl_sync(full, v, src, LN); };  // component src of this cell

    AdjLaneConsts<N, R, kRegs> cm;
    cm.init(k, rr, smc);
    const R b_r = k.b[rr], w_r = k.w[rr];

    // adjoint state of the cell: E and H (every lane keeps the copy lane 0 computes), row r of d
    R ebar = loaded ? a.Ea[ii] : R(0);
    R hbar = loaded ? a.Ha[ii] : R(0);
    R sbar = mrow ? a.Sa[r * a.stride + m] : R(0);
    R ebar_mur = before_mur ? a.Ea[n - 1] : R(0);  // the Mur cell's Ebar, kept by cell n - 2
    // this lane's rows of the outer-product gradients, summed over the launch
    R gDl[D], gT[2 * Q];
#pragma unroll
    for (int c = 0; c < D; ++c) gDl[c] = R(0);
#pragma unroll
    for (int c = 0; c < 2 * Q; ++c) gT[c] = R(0);
    R gb = R(0), gw = R(0), gc = R(0), gth = R(0);
    double gJ = 0.0;
    __syncthreads();  // padded constants in place

    for (int s = 0; s < a.nsteps; ++s) {
        const int j = a.j_hi - s;
        const unsigned char *f0 = a.rec + static_cast<int64_t>(j) * a.rec_set, *f1 = f0 + a.rec_set;
        const R *S0 = reinterpret_cast<const R *>(f0);
        const R *E0 = reinterpret_cast<const R *>(f0 + a.off_E), *E1 = reinterpret_cast<const R *>(f1 + a.off_E);
        // adjoint of E^{n+1} with the objective's term; the source's adjoint
        R ebn = ebar;
        if (is_probe) {
            const R e1 = E1[ii];
            ebn += jdt * e1;
            if (interior && r == 0) gJ += a.dt * static_cast<double>(e1) * static_cast<double>(e1);
        }
        if (is_src && interior && r == 0) a.dsrc[j] = static_cast<double>(ebn);
        // m: the Mur cell's adjoint (cell n - 2 only)
        R mbar = R(0);
        if (before_mur) {
            R em = ebar_mur;
            if (a.probe_cell == n - 1) em += jdt * E1[n - 1];
            mbar = (hard_src && a.source_cell == n - 1) ? R(0) : em;
        }
        R epre = R(0);
        if (in_e) {
            epre = (hard_src && is_src) ? R(0) : ebn;
            if (before_mur) epre += a.kappa * mbar;
        }
        if (r == 0) sEp[lc] = epre;
        __syncthreads();
        // Hbar^{n-1/2} of this cell
        const R ep_p = has_p ? sEp[lc + 1] : R(0);
        const R hh = hbar + (in_h ? cbdx * (epre - ep_p) : R(0));
        if (r == 0) sHh[lc] = hh;

        // the medium: forward recompute of the cell, then its reverse
        const R e = loaded ? E0[ii] : R(0);
        const R d = mrow ? S0[r * a.stride + m] : R(0);
        R y;  // y = d + (Dl d + b)
        {
            R acc = b_r;
#pragma unroll
            for (int c = 0; c < D; ++c) acc = fma(cm.dl_row(c), get(d, c), acc);
            y = d + acc;
        }
        R z;  // z = T^T y
        {
            R acc = cm.t_col(0) * get(y, 0);
#pragma unroll
            for (int c = 1; c < D; ++c) acc = fma(cm.t_col(c), get(y, c), acc);
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
            R acc = cm.t_row(0) * get(dz, 0);
#pragma unroll
            for (int c = 1; c < D; ++c) acc = fma(cm.t_row(c), get(dz, c), acc);
            y2 = y + acc;
        }
        R dn;  // dn = y2 + (Dl y2 + b)
        {
            R acc = b_r;
#pragma unroll
            for (int c = 0; c < D; ++c) acc = fma(cm.dl_row(c), get(y2, c), acc);
            dn = y2 + acc;
        }
        R dv = d, yv = y, zv = z, y2v = y2, dnv = dn, dzv = dz;
        if (!mrow) dv = yv = zv = y2v = dnv = dzv = R(0);
        const R pbar = (medium && in_e) ? -a.cb * epre : R(0);
        const R dnb = sbar + pbar * w_r;
        R y2b;  // y2b = dnb + Dl^T dnb
        {
            R acc = dnb;
#pragma unroll
            for (int c = 0; c < D; ++c) acc = fma(cm.dl_col(c), get(dnb, c), acc);
            y2b = acc;
        }
        R zb;  // zb = T^T y2b
        {
            R acc = cm.t_col(0) * get(y2b, 0);
#pragma unroll
            for (int c = 1; c < D; ++c) acc = fma(cm.t_col(c), get(y2b, c), acc);
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
            R acc = cm.t_row(0) * get(dzb, 0);
#pragma unroll
            for (int c = 1; c < D; ++c) acc = fma(cm.t_row(c), get(dzb, c), acc);
            yb = y2b + acc;
        }
        R db;  // db = yb + Dl^T yb
        {
            R acc = yb;
#pragma unroll
            for (int c = 0; c < D; ++c) acc = fma(cm.dl_col(c), get(yb, c), acc);
            db = acc;
        }
        // this lane's rows of the gradients (shuffles for every lane)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const R y2c = get(y2v, c), dc = get(dv, c);
            if (mrow) gDl[c] = fma(dnb, y2c, fma(yb, dc, gDl[c]));
        }
#pragma unroll
        for (int c = 0; c < 2 * Q; ++c) {
            const R dzc = get(dzv, c), dzbc = get(dzb, c);
            if (mrow) gT[c] = fma(y2b, dzc, fma(yv, dzbc, gT[c]));
        }
        if (mrow) {
            gb += dnb + yb;
            gw = fma(pbar, dnv, gw);
            sbar = db;
        }
        if (medium && r == 0) gc += pbar;
        if (medium && r < 2 * Q && r % 2 == 0) gth = fma(br, e * static_cast<R>(a.dt), gth);
        __syncthreads();  // Hbar of every cell in place
        // Ebar^n of this cell
        R eb = R(0);
        if (loaded) {
            const R hh_m = has_m ? sHh[lc - 1] : R(0);
            eb = (in_e ? a.ca * epre : R(0)) + a.ch * ((has_m && (periodic || ii - 1 <= n - 2) ? hh_m : R(0)) -
                                                        (in_h ? hh : R(0)));
            if (medium) eb += e_term;
            if (!periodic) {
                if (ii == 0 && !(hard_src && a.source_cell == 0)) eb += ebn;  // held: E^{n+1}_0 = E^n_0
                if (ii == n - 2) eb += mbar;                                // E^n_{n-2} in the Mur rule
                if (ii == n - 1) {                                          // E^n_{n-1} in the Mur rule
                    R em = ebn;
                    eb -= a.kappa * ((hard_src && a.source_cell == n - 1) ? R(0) : em);
                }
            }
        }
        ebar = eb;
        hbar = hh;
        if (before_mur) ebar_mur = a.ch * hh - a.kappa * mbar;
        // the next step's sEp / sHh writes come after its first barrier's reads of
        // sEp and this step's reads of sHh: the first barrier of the next step
        // orders them (sHh is written only after that barrier)
    }

    if (interior) {
        if (r == 0) {
            a.Eb[ii] = ebar;
            a.Hb[ii] = hbar;
        }
        if (mrow) {
            a.Sb[r * a.stride + m] = sbar;
#pragma unroll
            for (int c = 0; c < D; ++c) acc_add(a.acc, n, ii, L::Dl + r * D + c, static_cast<double>(gDl[c]));
#pragma unroll
            for (int c = 0; c < 2 * Q; ++c) acc_add(a.acc, n, ii, L::T + r * D + c, static_cast<double>(gT[c]));
            acc_add(a.acc, n, ii, L::b + r, static_cast<double>(gb));
            acc_add(a.acc, n, ii, L::w + r, static_cast<double>(gw));
        }
        if (medium && r == 0) acc_add(a.acc, n, ii, L::c, static_cast<double>(gc));
        if (medium && r < 2 * Q && r % 2 == 0) acc_add(a.acc, n, ii, L::th + r / 2, static_cast<double>(gth));
        if (r == 0 && is_probe) acc_add(a.acc, n, ii, L::J, gJ);
    }
}

}  // namespace mln
