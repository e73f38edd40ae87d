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

// Accumulator layout (entries of 8 bytes): Dl_bar (D x D) | b_bar (D) | w_bar (D) | c_bar |
// T_bar (D x D) | theta_bar (q) | J
template <int N>
struct AccLayout {
    static constexpr int D = Dims<N>::D, Q = Dims<N>::Q;
    static constexpr int Dl = 0, b = D * D, w = b + D, c = w + D, T = c + 1, th = T + D * D, J = th + Q,
                         size = J + 1;
};

// Each cell owns one column of the accumulators and adds to it at every
// launch (no atomics, no shuffles); mln_adjoint_reduce sums over the cells.
// FP64 contexts: one double per entry.
__device__ __forceinline__ void acc_add(double *acc, int64_t n, int64_t i, int idx, double v) {
    acc[idx * n + i] += v;
}
// FP32 contexts: a pair (hi, lo) of floats per entry in the same 8 bytes,
// summed by Knuth's two-sum (hi + lo holds the running sum to about twice
// the FP32 precision), so that the sweep does no FP64 arithmetic (1/64 of
// the FP32 rate on this GPU).
__device__ __forceinline__ void acc_add(float2 *acc, int64_t n, int64_t i, int idx, float v) {
    float2 a = acc[idx * n + i];
    const float s = a.x + v;
    const float bv = s - a.x;
    const float err = (a.x - (s - bv)) + (v - bv);
    a.x = s;
    a.y += err;
    acc[idx * n + i] = a;
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

// acc_add for NR entries of one cell: every entry read before any is written.
template <int NR>
__device__ __forceinline__ void acc_add_rows(double *acc, int64_t n, int64_t i, const int (&idx)[NR],
                                             const double (&v)[NR]) {
    double old[NR];
#pragma unroll
    for (int e = 0; e < NR; ++e) old[e] = acc[idx[e] * n + i];
#pragma unroll
    for (int e = 0; e < NR; ++e) acc[idx[e] * n + i] = old[e] + v[e];
}
template <int NR>
__device__ __forceinline__ void acc_add_rows(double *acc_d, int64_t n, int64_t i, const int (&idx)[NR],
                                             const float (&v)[NR]) {
    float2 *acc = reinterpret_cast<float2 *>(acc_d);
    float2 old[NR];
#pragma unroll
    for (int e = 0; e < NR; ++e) old[e] = acc[idx[e] * n + i];
#pragma unroll
    for (int e = 0; e < NR; ++e) {  // two-sum, as acc_add
        const float s = old[e].x + v[e];
        const float bv = s - old[e].x;
        const float err = (old[e].x - (s - bv)) + (v[e] - bv);
        acc[idx[e] * n + i] = make_float2(s, old[e].y + err);
    }
}

// The same sum over (hi, lo) pairs (FP32 contexts), in FP64.
__global__ void __launch_bounds__(256) mln_adjoint_reduce_pairs(const float2 *__restrict__ acc, int64_t n,
                                                                double *__restrict__ out) {
    __shared__ double part[256];
    const int k = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 a = acc[k * n + i];
        s += static_cast<double>(a.x) + static_cast<double>(a.y);
    }
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
    int64_t off_I;             // offset of step j's traced intermediates (StrangTraceCell rows) in set j
    int32_t j_hi, nsteps, halo, tile;
    const R *Ea, *Ha, *Sa;     // adjoints after step j_hi (of E^{n+1}, H^{n+1/2}, d^{n+1/2})
    R *Eb, *Hb, *Sb;           // adjoints before step j_hi - nsteps + 1
    double *dsrc;              // adjoint of the source sample of segment step j at dsrc[j], or nullptr
    double *acc;               // per-cell accumulators: entry k of cell i at k * n_cells + i (AccLayout;
                               // FP32 contexts: a float2 two-sum pair in each 8-byte entry)
    int64_t n_cells, mb, me, stride, source_cell, probe_cell;
    int32_t source_kind, boundary;  // boundary: 0 ring, 1 open (held cell 0, Mur at n - 1)
    double dt;
    R ch, ca, cb, inv_dx, kappa;
};

// The constant matrices as one lane needs them (its row r and column r of Dl
// and T): read from a padded copy in shared memory (rows of D + 1 entries:
// conflict-free for rows and columns), which leaves the registers to the
// accumulators (in FP32 the copy in registers had left the kernel at 126
// registers a thread and 8 % slower).
template <int N, typename R>
struct AdjLaneConsts {
    static constexpr int D = Dims<N>::D, P = D + 1, kMats = 2;
    const R *dl, *t;  // shared memory, [D][D + 1] each
    int rr;
    // block-cooperative: copy the matrices into the padded layout (needs a barrier after)
    __device__ __forceinline__ void init(const AdjConsts<N, R> &k, int r, R *sm) {
        for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
            const int o = (e / D) * P + e % D;
            sm[o] = k.Dl[e];
            sm[D * P + o] = k.T[e];
        }
        dl = sm;
        t = sm + D * P;
        rr = r;
    }
    __device__ __forceinline__ R dl_col(int j) const { return dl[j * P + rr]; }
    __device__ __forceinline__ R t_row(int j) const { return t[rr * P + j]; }
    __device__ __forceinline__ R t_col(int j) const { return t[j * P + rr]; }
};

// Most threads of a reverse-sweep block: FP32 up to 640 (80 cells of 8 lanes,
// the register file at ~100 registers a thread), FP64 512.
template <typename R>
struct AdjThreads {
    static constexpr int kMax = sizeof(R) == 4 ? 640 : 512;
};

// Vectors of a step that the lanes of a cell exchange through shared memory
// (one slot each, written once per step).
enum AdjSlot { kSlotD, kSlotDz, kSlotY2, kSlotDnb, kSlotY2b, kSlotDzb, kSlotYb, kSlotBr, kAdjSlots };

// Shared memory of the blocked reverse kernel: the padded constants,
// two field arrays of the block's cells and the exchange slots.
template <int N, typename R>
__host__ __device__ constexpr size_t adj_block_smem(int cells) {
    return AdjLaneConsts<N, R>::kMats * Dims<N>::D * (Dims<N>::D + 1) * sizeof(R) +
           2 * static_cast<size_t>(cells) * sizeof(R) +
           static_cast<size_t>(kAdjSlots) * cells * AdjLanes<N>::value * sizeof(R);
}

// The exchange of a vector held one component per lane: lane r of a cell
// stores its component in the cell's row of a slot, the warp synchronises,
// and every lane of the cell reads the whole row with 16-byte loads (the
// cell's lanes lie in one warp; rows are LN components, 16-byte aligned).
template <int LN>
__device__ __forceinline__ void adj_row_load(const float *p, float (&v)[LN]) {
#pragma unroll
    for (int i = 0; i < LN / 4; ++i) {
        const float4 t = reinterpret_cast<const float4 *>(p)[i];
        v[4 * i] = t.x;
        v[4 * i + 1] = t.y;
        v[4 * i + 2] = t.z;
        v[4 * i + 3] = t.w;
    }
}
template <int LN>
__device__ __forceinline__ void adj_row_load(const double *p, double (&v)[LN]) {
#pragma unroll
    for (int i = 0; i < LN / 2; ++i) {
        const double2 t = reinterpret_cast<const double2 *>(p)[i];
        v[2 * i] = t.x;
        v[2 * i + 1] = t.y;
    }
}

// The temporally blocked reverse sweep with one lane per component: the
// AdjLanes lanes of a cell each own one row r < D of every vector and of
// every product and read the other components of a product's input from
// the cell's row of an exchange slot in shared memory (each vector stored
// once, read back whole). The step's forward values d', z, d'' (and in FP64
// the plane terms) come from the recomputation's trace (StrangTraceCell) and
// d^{n+1/2} from the next recorded state, so only the transposed products run here;
// each lane also owns row r of the
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
__global__ void __launch_bounds__(AdjThreads<R>::kMax) mln_adjoint_block(const __grid_constant__ AdjBlockArgs<R> a,
                                                         const __grid_constant__ AdjConsts<N, R> k) {
    constexpr int D = Dims<N>::D, Q = Dims<N>::Q, LN = AdjLanes<N>::value;
    using L = AccLayout<N>;
    extern __shared__ __align__(16) unsigned char adj_smem[];
    R *smc = reinterpret_cast<R *>(adj_smem);
    const int cells = blockDim.x / LN;
    R *sEp = smc + AdjLaneConsts<N, R>::kMats * D * (D + 1);  // epre of each cell
    R *sHh = sEp + cells;                            // new Hbar of each cell
    R *sVec = sHh + cells;                           // exchange slots, [kAdjSlots][cells][LN]

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
    // store this lane's component of a vector in its slot; read a slot's row
    auto stage = [&](int sl, R v) { sVec[(sl * cells + lc) * LN + r] = v; };
    auto put = [&](int sl, R v) {
        stage(sl, v);
        __syncwarp();
    };
    auto row = [&](int sl, R (&v)[LN]) { adj_row_load<LN>(sVec + (sl * cells + lc) * LN, v); };

    AdjLaneConsts<N, R> cm;
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
    // The recorded forward values of step j: E^j (E^{j+1} at the probe), this
    // lane's row of d^j, of the traced intermediates y = d', z = T^T d' (plane
    // rows) and y2 = d'', and of dn = d^{j+1}; loaded one step ahead, so that
    // the loads' latency is spent under the previous step (dn is the previous
    // step's d).
    auto rec_S = [&](int jj) { return reinterpret_cast<const R *>(a.rec + static_cast<int64_t>(jj) * a.rec_set); };
    auto rec_E = [&](int jj) {
        return reinterpret_cast<const R *>(a.rec + static_cast<int64_t>(jj) * a.rec_set + a.off_E);
    };
    auto rec_I = [&](int jj, int rowi) {
        return reinterpret_cast<const R *>(a.rec + static_cast<int64_t>(jj) * a.rec_set + a.off_I)[rowi * a.stride + m];
    };
    const bool zrow = mrow && r < 2 * Q;
    R e_nx = loaded ? rec_E(a.j_hi)[ii] : R(0);
    R d_nx = mrow ? rec_S(a.j_hi)[r * a.stride + m] : R(0);
    R e1_nx = is_probe ? rec_E(a.j_hi + 1)[ii] : R(0);
    R y_nx = mrow ? rec_I(a.j_hi, r) : R(0);
    R z_nx = zrow ? rec_I(a.j_hi, D + r) : R(0);
    R y2_nx = mrow ? rec_I(a.j_hi, D + 2 * Q + r) : R(0);
    R dn_nx = mrow ? rec_S(a.j_hi + 1)[r * a.stride + m] : R(0);
    // FP64: this lane's plane (r / 2), its sin phi and cos phi - 1 recorded
    // too (their evaluation is a quarter of the step's FP64 work); FP32
    // evaluates them (fewer loads on its latency-bound path: measured faster)
    constexpr bool kRecPlanes = sizeof(R) == 8;
    R sn_nx = (kRecPlanes && zrow) ? rec_I(a.j_hi, 2 * D + 2 * Q + r / 2) : R(0);
    R c1_nx = (kRecPlanes && zrow) ? rec_I(a.j_hi, 2 * D + 3 * Q + r / 2) : R(0);
    __syncthreads();  // padded constants in place

    for (int s = 0; s < a.nsteps; ++s) {
        const int j = a.j_hi - s;
        const R *E1 = rec_E(j + 1);
        const R e = e_nx, d = d_nx, e1_rec = e1_nx, y = y_nx, z = z_nx, y2 = y2_nx, dn = dn_nx;
        R snp = sn_nx, c1p = c1_nx;
        if (s + 1 < a.nsteps) {
            e_nx = loaded ? rec_E(j - 1)[ii] : R(0);
            d_nx = mrow ? rec_S(j - 1)[r * a.stride + m] : R(0);
            e1_nx = e;  // E^{j} of this cell is E^{(j-1)+1}
            y_nx = mrow ? rec_I(j - 1, r) : R(0);
            z_nx = zrow ? rec_I(j - 1, D + r) : R(0);
            y2_nx = mrow ? rec_I(j - 1, D + 2 * Q + r) : R(0);
            dn_nx = d;  // d^{j} is the dn of step j - 1
            if constexpr (kRecPlanes) {
                sn_nx = zrow ? rec_I(j - 1, 2 * D + 2 * Q + r / 2) : R(0);
                c1_nx = zrow ? rec_I(j - 1, 2 * D + 3 * Q + r / 2) : R(0);
            }
        }
        // adjoint of E^{n+1} with the objective's term; the source's adjoint
        R ebn = ebar;
        if (is_probe) {
            const R e1 = e1_rec;
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

        // the medium: the step's forward values (recorded), then its reverse
        R v[LN];
        if constexpr (!kRecPlanes) {
            R sn[Q], c1[Q];
            plane_terms<N>(k.psi_dt, e, sn, c1);
            // this lane's plane terms, selected in registers (no indexed array)
            c1p = c1[0];
            snp = sn[0];
#pragma unroll
            for (int q = 1; q < Q; ++q)
                if (rr / 2 == q) {
                    c1p = c1[q];
                    snp = sn[q];
                }
        }
        const R z_pair = __shfl_xor_sync(full, z, 1, LN);
        R dz = R(0);  // (R - I) z
        if (r < 2 * Q) dz = (r % 2 == 0) ? fma(c1p, z, snp * z_pair) : fma(c1p, z, -(snp * z_pair));
        // d, dz and y2 for the gradients' outer products
        stage(kSlotD, d);
        stage(kSlotDz, dz);
        stage(kSlotY2, y2);
        __syncwarp();
        R yv = y, zv = z, dnv = dn;
        if (!mrow) yv = zv = dnv = R(0);
        const R pbar = (medium && in_e) ? -a.cb * epre : R(0);
        const R dnb = sbar + pbar * w_r;
        R y2b, zb;
        put(kSlotDnb, dnb);
        row(kSlotDnb, v);
        {  // y2b = dnb + Dl^T dnb
            R acc = dnb;
#pragma unroll
            for (int c = 0; c < D; ++c) acc = fma(cm.dl_col(c), v[c], acc);
            y2b = acc;
        }
        {  // zb = T^T y2b
            put(kSlotY2b, y2b);
            row(kSlotY2b, v);
            R acc = cm.t_col(0) * v[0];
#pragma unroll
            for (int c = 1; c < D; ++c) acc = fma(cm.t_col(c), v[c], acc);
            zb = acc;
        }
        const R zb_pair = __shfl_xor_sync(full, zb, 1, LN);
        const R zv_pair = __shfl_xor_sync(full, zv, 1, LN);
        R dzb = R(0), br = R(0);
        if (r < 2 * Q) {
            const bool even = r % 2 == 0;
            dzb = even ? fma(c1p, zb, -(snp * zb_pair)) : fma(c1p, zb, snp * zb_pair);
            if (even) {
                const R zx = zv, zy = zv_pair, bx = zb, by = zb_pair, cs = R(1) + c1p;
                br = bx * fma(-snp, zx, cs * zy) + by * fma(-cs, zx, -(snp * zy));
            }
        }
        R e_term = R(0);
        stage(kSlotBr, br);
        stage(kSlotDzb, dzb);
        __syncwarp();
        row(kSlotBr, v);
#pragma unroll
        for (int p = 0; p < Q; ++p) e_term = fma(k.theta_dt[p], v[2 * p], e_term);
        row(kSlotDzb, v);
        R yb, db;
        {  // yb = y2b + T dzb
            R acc = cm.t_row(0) * v[0];
#pragma unroll
            for (int c = 1; c < D; ++c) acc = fma(cm.t_row(c), v[c], acc);
            yb = y2b + acc;
        }
        {  // db = yb + Dl^T yb
            put(kSlotYb, yb);
            row(kSlotYb, v);
            R acc = yb;
#pragma unroll
            for (int c = 0; c < D; ++c) acc = fma(cm.dl_col(c), v[c], acc);
            db = acc;
        }
        // this lane's rows of the gradients, from the slots of y2, d, dz and dzb
        // (a lane with mrow belongs to a medium cell, whose rows c < D hold them)
        if (mrow) {
            R w2[LN];
            row(kSlotY2, v);
            row(kSlotD, w2);
#pragma unroll
            for (int c = 0; c < D; ++c) gDl[c] = fma(dnb, v[c], fma(yb, w2[c], gDl[c]));
            row(kSlotDz, v);
            row(kSlotDzb, w2);
#pragma unroll
            for (int c = 0; c < 2 * Q; ++c) gT[c] = fma(y2b, v[c], fma(yv, w2[c], gT[c]));
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
        // into the cell's accumulator column: doubles (FP64), two-sum pairs (FP32)
        auto add = [&](int idx, R v) {
            if constexpr (sizeof(R) == 8) acc_add(a.acc, n, ii, idx, v);
            else acc_add(reinterpret_cast<float2 *>(a.acc), n, ii, idx, v);
        };
        if (mrow) {
            a.Sb[r * a.stride + m] = sbar;
            // this lane's row entries: all loaded first, then added and stored (one
            // read-modify-write after another would wait a memory round trip each,
            // since the compiler cannot tell the entries apart)
            constexpr int NR = D + 2 * Q + 2;
            R v[NR];
            int idx[NR];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                v[c] = gDl[c];
                idx[c] = L::Dl + r * D + c;
            }
#pragma unroll
            for (int c = 0; c < 2 * Q; ++c) {
                v[D + c] = gT[c];
                idx[D + c] = L::T + r * D + c;
            }
            v[NR - 2] = gb;
            idx[NR - 2] = L::b + r;
            v[NR - 1] = gw;
            idx[NR - 1] = L::w + r;
            acc_add_rows<NR>(a.acc, n, ii, idx, v);
        }
        if (medium && r == 0) add(L::c, gc);
        if (medium && r < 2 * Q && r % 2 == 0) add(L::th + r / 2, gth);
        if (r == 0 && is_probe) {
            if constexpr (sizeof(R) == 8) {
                acc_add(a.acc, n, ii, L::J, gJ);
            } else {  // the FP64 partial sum as two floats
                const float hi = static_cast<float>(gJ);
                acc_add(reinterpret_cast<float2 *>(a.acc), n, ii, L::J, hi);
                acc_add(reinterpret_cast<float2 *>(a.acc), n, ii, L::J, static_cast<float>(gJ - static_cast<double>(hi)));
            }
        }
    }
}

}  // namespace mln
