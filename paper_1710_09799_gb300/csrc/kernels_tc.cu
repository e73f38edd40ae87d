// Tensor-core cell model (FP32 state, merged form, N = 5 and 6). The merged
// step (Eqs. 23, 25-26, 17)
//   z = T^T y,  dz = (R(phi) - I) z,  r = y + T dz,
//   y' = r + (A0^2 - I) r + A0 b + b,  dP/dt = (A0^T w) . r + c'
// is regrouped into two dense products per step,
//   z = T^T y                                                (before the rotation)
//   [y' - y ; dP/dt] = [C1, b2, A0^2 T ; wm^T, c', wm^T T] [y ; 1 ; dz]   (after it)
// with C1 = A0^2 - I, b2 = A0 b + b and wm = A0^T w (the constant offsets ride
// on a column of ones); the increment (second product) is added to y in FP32. Both run as tcgen05.mma kind::tf32 over 128 cells at a time,
// each FP32 operand split into a TF32 high and low part (three MMAs per K
// block: lo*hi + hi*lo + hi*hi, FP32 accumulation in tensor memory). The
// rotation, the FP32 additions and the FDTD update run on the FP32 pipe.
//
// A CTA holds four independent tiles of 128 cells (one warpgroup each, with
// its own K-cell halo on both sides, as in the temporal blocking of the other
// cell models); the warpgroups synchronise only among themselves, so the
// tensor core works for one tile while the others rotate and update fields.
// The CTA is persistent: the B operands (hi and lo images) are staged once in
// shared memory and the warpgroups loop over tiles. Each cell's row of y is
// written by its thread into tensor memory (tcgen05.st), where both products
// read it; its row of dz goes to shared memory.
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "setup.h"
#include "tc.cuh"
#include "tc_kernel.h"

namespace mln {

// Layout of one CTA of the tensor-core kernel for N levels.
template <int N>
struct TcShape {
    static constexpr int D = Dims<N>::D, Q = Dims<N>::Q, P = 2 * Q;
    static constexpr int KA = (D + 1 + 7) / 8 * 8;     // K over the state and the constant-1 column
    static constexpr int KP = (P + 7) / 8 * 8;         // K over the plane coordinates
    static constexpr int N1 = (P + 15) / 16 * 16;      // MMA N of z = T^T y
    static constexpr int N3 = (D + 1 + 15) / 16 * 16;  // MMA N of the increment and dP/dt
    static constexpr int L1 = (P + 7) / 8 * 8;         // accumulator columns read back
    static constexpr int L3 = (D + 1 + 7) / 8 * 8;
    static constexpr int G = 4;                        // warpgroups (tiles) per CTA
    static constexpr int ROWS = 128;
    // tensor-memory columns of one group: y hi | y lo | accumulator
    static constexpr int Y_HI = 0, Y_LO = KA, ACC = 2 * KA, GCOLS = 128;
    static constexpr uint32_t TMEM_COLS = static_cast<uint32_t>(G * GCOLS);
    // B images (hi, lo each): T^T (N1 x KA), [C1; wm^T] (N3 x KA), [A0^2 T; wm^T T] (N3 x KP)
    static constexpr int B1 = N1 * KA * 4, BY = N3 * KA * 4, BZ = N3 * KP * 4;
    static constexpr int BIMG = 2 * (B1 + BY + BZ);
    static constexpr int ZBYTES = ROWS * KP * 4;       // one dz image of a group
    static constexpr int OFF_Z = (BIMG + 127) / 128 * 128;
    static constexpr int OFF_E = OFF_Z + G * 2 * ZBYTES;
    static constexpr int OFF_H = OFF_E + G * ROWS * 4;
    static constexpr int OFF_BAR = OFF_H + G * ROWS * 4;
    static constexpr int SMEM = OFF_BAR + 8 * (G + 1) + 16;  // one MMA barrier per group, one for the B copy
    static_assert(ACC + (N1 > N3 ? N1 : N3) <= GCOLS, "tensor-memory columns of one group");
    static_assert(L1 <= N1 && L3 <= N3, "read-back beyond the accumulator");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

template <int N>
struct TcScalars {
    float psi_dt[N - 1];  // (m_a - m_{N-1}) dt / hbar: base angles per unit field
};

namespace {

// x = hi + lo exactly: hi is x rounded to TF32 (integer add and mask: the
// conversion instruction issues on a slower pipe), lo = x - hi in FP32, which
// the MMA reads as TF32 (its 13 low bits ignored), so hi + lo(TF32) = x up to
// 2^-21 |x|.
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    hi = tc::tf32_bits(__float_as_uint(x));
    lo = __float_as_uint(x - __uint_as_float(hi));
}

// Stage row `row` of an A operand from v[0..n), then `one` (1.0 at column n
// when set: the column that carries constant offsets through the product),
// zero-padded to kx columns (a multiple of 8): hi and lo TF32 parts. TA: into
// tensor memory at columns t_hi, t_lo of this thread's lane (t_* carry the
// warp's lane base); else into shared memory (hi image at a, lo image ABYTES
// later, layout K extent K).
template <bool TA, int K, int kx, int n, int ABYTES, bool one = false>
__device__ __forceinline__ void stage_row(unsigned char *a, uint32_t t_hi, uint32_t t_lo, int row, const float *v) {
    static_assert(n + (one ? 1 : 0) <= kx, "row longer than the staged width");
    auto split = [&](int k, uint32_t &h, uint32_t &l) {
        if (k < n) {
            split_tf32(v[k], h, l);
        } else {
            h = (one && k == n) ? 0x3F800000u : 0u;
            l = 0u;
        }
    };
    if constexpr (TA) {
#pragma unroll
        for (int c = 0; c < kx; c += 8) {
            uint32_t h[8], l[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) split(c + e, h[e], l[e]);
            tc::st_x8(t_hi + c, h);
            tc::st_x8(t_lo + c, l);
        }
        tc::st_wait();
    } else {
#pragma unroll
        for (int kg = 0; kg < kx / 4; ++kg) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) split(kg * 4 + e, h[e], l[e]);
            const int off = tc::core_offset(row, kg * 4, K);
            *reinterpret_cast<uint4 *>(a + off) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4 *>(a + ABYTES + off) = make_uint4(l[0], l[1], l[2], l[3]);
        }
        tc::fence_async_smem();
    }
}

// D = A B^T over K = kx, 3 x TF32 (lo*hi, hi*lo, hi*hi), issued by one thread.
// TA: a_hi, a_lo are tensor-memory addresses; else shared-memory addresses of
// A images with stride-dimension byte offset sbo_a.
template <bool TA, int kx>
__device__ __forceinline__ void issue_product(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t sbo_a,
                                              uint32_t b_hi, uint32_t b_lo, uint32_t sbo_b, uint32_t idesc) {
    auto mma = [&](uint32_t a, uint32_t b, int kb, uint32_t acc) {
        const uint64_t bd = tc::smem_desc(b + kb * 256, 128, sbo_b);
        if constexpr (TA)
            tc::mma_tf32_ts(d, a + kb * 8, bd, idesc, acc);
        else
            tc::mma_tf32(d, tc::smem_desc(a + kb * 256, 128, sbo_a), bd, idesc, acc);
    };
#pragma unroll
    for (int kb = 0; kb < kx / 8; ++kb) mma(a_lo, b_hi, kb, kb > 0 ? 1u : 0u);
#pragma unroll
    for (int kb = 0; kb < kx / 8; ++kb) mma(a_hi, b_lo, kb, 1u);
#pragma unroll
    for (int kb = 0; kb < kx / 8; ++kb) mma(a_hi, b_hi, kb, 1u);
}

// Read `cols` (multiple of 8) accumulator columns of this thread's lane.
template <int cols>
__device__ __forceinline__ void read_cols(uint32_t taddr, float (&v)[cols]) {
    constexpr int n32 = cols / 32;
#pragma unroll
    for (int c = 0; c < n32; ++c) {
        float t[32];
        tc::ld_x32(taddr + c * 32, t);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[c * 32 + i] = t[i];
    }
#pragma unroll
    for (int c = n32 * 32; c < cols; c += 8) {
        float t[8];
        tc::ld_x8(taddr + c, t);
#pragma unroll
        for (int i = 0; i < 8; ++i) v[c + i] = t[i];
    }
}

}  // namespace

template <int N>
__global__ void __launch_bounds__(512, 1)
    mln_tc_kernel(const __grid_constant__ BlockArgs<float> a, const __grid_constant__ TcScalars<N> k,
                  const uint4 *__restrict__ bimg, int64_t ntiles) {
    using S = TcShape<N>;
    constexpr int D = S::D, Q = S::Q, P = S::P, G = S::G, ROWS = S::ROWS;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, g = tid / ROWS, j = tid % ROWS, warp = tid / 32;
    unsigned char *sZ = smem + S::OFF_Z + g * 2 * S::ZBYTES;
    float *sE = reinterpret_cast<float *>(smem + S::OFF_E) + g * ROWS;
    float *sH = reinterpret_cast<float *>(smem + S::OFF_H) + g * ROWS;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S::OFF_BAR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + S::OFF_BAR + 8 * (G + 1));

    // B images: one bulk copy into shared memory, completion on bars[G]
    if (tid <= G) tc::mbar_init(tc::smem_addr(&bars[tid]), 1);
    tc::mbar_init_fence();
    __syncthreads();
    if (tid == 0) {
        tc::mbar_expect_tx(tc::smem_addr(&bars[G]), S::BIMG);
        tc::bulk_load(tc::smem_addr(smem), bimg, S::BIMG, tc::smem_addr(&bars[G]));
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_addr(tslot), S::TMEM_COLS);
        tc::tmem_relinquish();
    }
    bool ok = tc::mbar_wait(tc::smem_addr(&bars[G]), 0);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t tg = tmem + static_cast<uint32_t>(g * S::GCOLS);                // group's columns, lane 0
    const uint32_t lanes = static_cast<uint32_t>((warp % 4) * 32) << 16;          // this warp's lanes
    const uint32_t bar = tc::smem_addr(&bars[g]);
    const uint32_t y_hi = tg + S::Y_HI, y_lo = tg + S::Y_LO, acc = tg + S::ACC;
    const uint32_t z_hi = tc::smem_addr(sZ), z_lo = z_hi + S::ZBYTES;
    const uint32_t b1h = tc::smem_addr(smem), b1l = b1h + S::B1;
    const uint32_t byh = b1l + S::B1, byl = byh + S::BY;
    const uint32_t bzh = byl + S::BY, bzl = bzh + S::BZ;
    const uint32_t id1 = tc::idesc_tf32(S::N1), id3 = tc::idesc_tf32(S::N3);
    const int bar_id = 1 + g;
    uint32_t phase = 0;
    // descriptors of the first K block of each shared-memory operand (block kb
    // starts kb * 256 bytes later: 16 units further in the address field)
    const uint64_t d1h = tc::smem_desc(b1h, 128, S::KA * 32), d1l = tc::smem_desc(b1l, 128, S::KA * 32);
    const uint64_t dyh = tc::smem_desc(byh, 128, S::KA * 32), dyl = tc::smem_desc(byl, 128, S::KA * 32);
    const uint64_t dzh = tc::smem_desc(bzh, 128, S::KP * 32), dzl = tc::smem_desc(bzl, 128, S::KP * 32);
    const uint64_t dah = tc::smem_desc(z_hi, 128, S::KP * 32), dal = tc::smem_desc(z_lo, 128, S::KP * 32);

    // z = T^T y: A = y from tensor memory (one thread)
    auto issue_z = [&] {
#pragma unroll
        for (int kb = 0; kb < S::KA / 8; ++kb) tc::mma_tf32_ts(acc, y_lo + kb * 8, d1h + 16 * kb, id1, kb > 0);
#pragma unroll
        for (int kb = 0; kb < S::KA / 8; ++kb) tc::mma_tf32_ts(acc, y_hi + kb * 8, d1l + 16 * kb, id1, 1u);
#pragma unroll
        for (int kb = 0; kb < S::KA / 8; ++kb) tc::mma_tf32_ts(acc, y_hi + kb * 8, d1h + 16 * kb, id1, 1u);
    };
    // [increment ; dP/dt - c'] = [C1, A0^2 T ; wm^T, wm^T T] [y ; dz]: y from
    // tensor memory, dz from shared memory (one thread)
    auto issue_inc = [&] {
        auto part = [&](uint32_t ya, uint64_t yb, uint64_t za, uint64_t zb, bool first) {
#pragma unroll
            for (int kb = 0; kb < S::KA / 8; ++kb)
                tc::mma_tf32_ts(acc, ya + kb * 8, yb + 16 * kb, id3, (first && kb == 0) ? 0u : 1u);
#pragma unroll
            for (int kb = 0; kb < S::KP / 8; ++kb) tc::mma_tf32(acc, za + 16 * kb, zb + 16 * kb, id3, 1u);
        };
        part(y_lo, dyh, dal, dzh, true);
        part(y_hi, dyl, dah, dzl, false);
        part(y_hi, dyh, dah, dzh, false);
    };
    // one elected lane of the group's first warp issues, from a converged warp
    const bool mma_warp = warp % 4 == 0;
    auto issue = [&](auto f) {
        if (mma_warp) {
            if (tc::elect_one()) {
                tc::fence_after_sync();
                f();
                tc::mma_commit(bar);
            }
            __syncwarp();
        }
    };
    auto wait = [&] {
        ok = tc::mbar_wait(bar, phase) && ok;
        phase ^= 1;
        tc::fence_after_sync();
    };

    const int64_t n = a.n_cells;
    const bool periodic = a.boundary == 0;
    for (int64_t tile_index = static_cast<int64_t>(blockIdx.x) * G + g; tile_index < ntiles;
         tile_index += static_cast<int64_t>(gridDim.x) * G) {
        const int64_t t0 = tile_index * a.tile;
        const int64_t t1 = min(t0 + a.tile, n);
        // a tile that starts at the Mur cell loads one more cell on the left:
        // the Mur cell's value comes from its left neighbour's row in the same
        // step (that tile has one cell, so 2 halo + 2 <= 128 rows)
        const int lh = a.halo + ((!periodic && t0 == n - 1) ? 1 : 0);
        const int L = static_cast<int>(t1 - t0) + lh + a.halo;
        const int64_t gi = t0 - lh + j;
        int64_t gm = gi;
        bool loaded = j < L;
        if (periodic) {
            gm = wrap_index(gi, n);
        } else {
            loaded = loaded && gi >= 0 && gi < n;
        }
        const bool medium = loaded && gm >= a.mb && gm < a.me;
        const int64_t m = gm - a.mb;
        float y[D];
#pragma unroll
        for (int i = 0; i < D; ++i) y[i] = medium ? a.s_in[i * a.stride + m] : 0.0f;
        float e = loaded ? a.E_in[gm] : 0.0f;
        float h = loaded ? a.H_in[gm] : 0.0f;
        sE[j] = e;
        sH[j] = h;
        const bool h_upd = loaded && (j + 1 < L) && (periodic || gm < n - 1);
        const bool e_upd = loaded && j >= 1 && (periodic || (gm > 0 && gm < n - 1));
        const bool mur = !periodic && loaded && gm == n - 2 && j + 1 < L;
        const bool is_src = a.src != nullptr && loaded && gm == a.source_cell;
        stage_row<true, S::KA, S::KA, D, 0, true>(nullptr, y_hi + lanes, y_lo + lanes, j, y);
        tc::fence_before_sync();
        tc::bar_sync(bar_id, ROWS);
        if (a.nsteps > 0) issue(issue_z);

        for (int st = 0; st < a.nsteps; ++st) {
            if (h_upd) {
                h = fma(a.ch, sE[j + 1] - e, h);
                sH[j] = h;
            }
            wait();
            float z[S::L1];
            read_cols<S::L1>(acc + lanes, z);
            tc::ld_wait();
            // dz = (R(phi) - I) z with phi from E^n; zero for cells without medium
            float dz[P];
            {
                float sn[Q], c1[Q];
                plane_terms<N>(k.psi_dt, e, sn, c1);
#pragma unroll
                for (int p = 0; p < Q; ++p) {
                    dz[2 * p] = medium ? fma(c1[p], z[2 * p], sn[p] * z[2 * p + 1]) : 0.0f;
                    dz[2 * p + 1] = medium ? fma(c1[p], z[2 * p + 1], -(sn[p] * z[2 * p])) : 0.0f;
                }
            }
            stage_row<false, S::KP, S::KP, P, S::ZBYTES>(sZ, 0, 0, j, dz);
            tc::fence_before_sync();
            tc::bar_sync(bar_id, ROWS);  // dz staged, H^{n+1/2} published
            issue(issue_inc);
            wait();
            float dpdt;
            {
                float d3[S::L3];
                read_cols<S::L3>(acc + lanes, d3);
                tc::ld_wait();
#pragma unroll
                for (int i = 0; i < D; ++i) y[i] = medium ? y[i] + d3[i] : 0.0f;
                dpdt = medium ? d3[D] : 0.0f;
            }
            float en = e;
            if (e_upd) en = fma(a.ca, e, a.cb * fma(h - sH[j - 1], a.inv_dx, -dpdt));
            float e_mur = 0.0f;
            if (mur) e_mur = fma(a.kappa, en - sE[j + 1], e);
            if (is_src) {
                const float v = static_cast<float>(a.src[st]);
                en = (a.source_kind == 1) ? v : en + v;
            }
            if (mur) {
                if (a.src != nullptr && a.source_cell == n - 1) {
                    const float v = static_cast<float>(a.src[st]);
                    e_mur = (a.source_kind == 1) ? v : e_mur + v;
                }
                sE[j + 1] = e_mur;
            }
            e = en;
            if (loaded && !(!periodic && gm == n - 1)) sE[j] = e;
            stage_row<true, S::KA, S::KA, D, 0, true>(nullptr, y_hi + lanes, y_lo + lanes, j, y);
            tc::fence_before_sync();
            tc::bar_sync(bar_id, ROWS);  // E^{n+1} published, y staged for the next step
            if (!periodic && loaded && gm == n - 1) e = sE[j];
            if (st + 1 < a.nsteps) issue(issue_z);
        }

        const bool interior = loaded && j >= lh && j < lh + static_cast<int>(t1 - t0);
        if (interior) {
            a.E_out[gm] = e;
            a.H_out[gm] = h;
            if (medium) {
#pragma unroll
                for (int i = 0; i < D; ++i) a.s_out[i * a.stride + m] = y[i];
            }
            if (!isfinite(e)) atomicOr(a.flags, 1u);
        }
        tc::bar_sync(bar_id, ROWS);  // sE / sH are reused by the next tile
    }
    if (!ok) atomicOr(a.flags, 2u);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, S::TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------
// Diagnostic product C = A B^T (A: 128 x KC, B: NC x KC) through the same
// staging, split and issue path as the step kernel (one warpgroup).
// ISSUE = false leaves the MMA and its commit out: nothing arrives on the
// mbarrier, and the bounded completion wait runs out (the timeout path).
template <int NC, int KC, bool TA, bool ISSUE = true>
__global__ void __launch_bounds__(128, 1)
    mln_tc_product_kernel(const float *__restrict__ A, const uint4 *__restrict__ bimg, float *__restrict__ C,
                          unsigned int *flag) {
    constexpr int ABYTES = TA ? 0 : 128 * KC * 4, BBYTES = NC * KC * 4;
    constexpr uint32_t COLS = 256;  // A hi, A lo (TA) and the accumulator
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *sB = smem;                       // hi, lo
    unsigned char *sA = smem + 2 * BBYTES;          // hi, lo (shared-memory A only)
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * BBYTES + 2 * ABYTES);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    const int j = threadIdx.x, warp = j / 32;
    for (int o = j; o < 2 * BBYTES / 16; o += 128) reinterpret_cast<uint4 *>(sB)[o] = bimg[o];
    if (j == 0) tc::mbar_init(tc::smem_addr(bar), 1);
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_addr(tslot), COLS);
        tc::tmem_relinquish();
    }
    tc::mbar_init_fence();
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t lane = static_cast<uint32_t>(warp * 32) << 16;
    const uint32_t acc = tmem + (TA ? 2 * KC : 0);
    float v[KC];
#pragma unroll
    for (int i = 0; i < KC; ++i) v[i] = A[j * KC + i];
    stage_row<TA, KC, KC, KC, ABYTES>(sA, tmem + lane, tmem + KC + lane, j, v);
    tc::fence_before_sync();
    __syncthreads();
    if (ISSUE && j == 0) {
        tc::fence_after_sync();
        const uint32_t ah = TA ? tmem : tc::smem_addr(sA), al = TA ? tmem + KC : ah + ABYTES;
        const uint32_t bh = tc::smem_addr(sB);
        issue_product<TA, KC>(acc, ah, al, KC * 32, bh, bh + BBYTES, KC * 32, tc::idesc_tf32(NC));
        tc::mma_commit(tc::smem_addr(bar));
    }
    const bool ok = tc::mbar_wait(tc::smem_addr(bar), 0);
    tc::fence_after_sync();
    float c[NC];
    read_cols<NC>(acc + lane, c);
    tc::ld_wait();
#pragma unroll
    for (int i = 0; i < NC; ++i) C[j * NC + i] = c[i];
    if (!ok) atomicOr(flag, 1u);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, COLS);
    }
}

// ---------------------------------------------------------------------------
// Host side.

namespace {

void split_tf32(double x, float &hi, float &lo) {
    uint32_t b;
    float f = static_cast<float>(x);
    std::memcpy(&b, &f, 4);
    b = tc::tf32_bits(b);
    std::memcpy(&hi, &b, 4);
    float r = static_cast<float>(x - static_cast<double>(hi));
    std::memcpy(&b, &r, 4);
    b = tc::tf32_bits(b);
    std::memcpy(&lo, &b, 4);
}

// hi and lo images of an R x K operand whose entry (r, k) is f(r, k)
// (zero outside rows x cols), appended to out.
template <typename F>
void append_image(std::vector<unsigned char> &out, int R, int K, F f) {
    std::vector<unsigned char> hi(static_cast<size_t>(R) * K * 4, 0), lo(hi.size(), 0);
    for (int r = 0; r < R; ++r)
        for (int k = 0; k < K; ++k) {
            float h, l;
            split_tf32(f(r, k), h, l);
            std::memcpy(hi.data() + tc::core_offset(r, k, K), &h, 4);
            std::memcpy(lo.data() + tc::core_offset(r, k, K), &l, 4);
        }
    out.insert(out.end(), hi.begin(), hi.end());
    out.insert(out.end(), lo.begin(), lo.end());
}

template <int N>
void pack_tc_t(const Setup &s, double dt, std::vector<unsigned char> &img, std::vector<unsigned char> &scal) {
    using S = TcShape<N>;
    constexpr int D = S::D, P = S::P;
    // A0^2 T = T + C1 T and wm^T T, in FP64
    std::vector<double> A2T(static_cast<size_t>(D) * P), wT(P);
    for (int i = 0; i < D; ++i)
        for (int p = 0; p < P; ++p) {
            double acc = s.T[i * D + p];
            for (int l = 0; l < D; ++l) acc += s.C1[i * D + l] * s.T[l * D + p];
            A2T[i * P + p] = acc;
        }
    for (int p = 0; p < P; ++p) {
        double acc = 0.0;
        for (int i = 0; i < D; ++i) acc += s.wm[i] * s.T[i * D + p];
        wT[p] = acc;
    }
    img.clear();
    // B1 (N1 x KA): row p, column k = T[k][p] (plane columns p < P; zero at the constant column)
    append_image(img, S::N1, S::KA, [&](int p, int k) { return (p < P && k < D) ? s.T[k * D + p] : 0.0; });
    // BY (N3 x KA): rows i < D = [C1 | b2] (C1 = A0^2 - I, b2 = A0 b + b at the
    // constant column D), row D = [wm | c'] (wm = A0^T w)
    append_image(img, S::N3, S::KA, [&](int i, int k) {
        if (k > D) return 0.0;
        if (i < D) return k < D ? s.C1[i * D + k] : s.b2[i];
        if (i == D) return k < D ? s.wm[k] : s.cm;
        return 0.0;
    });
    // BZ (N3 x KP): rows i < D = A0^2 T (plane columns), row D = wm^T T
    append_image(img, S::N3, S::KP, [&](int i, int p) {
        if (p >= P) return 0.0;
        if (i < D) return A2T[i * P + p];
        return i == D ? wT[p] : 0.0;
    });
    TcScalars<N> t;
    std::memset(&t, 0, sizeof(t));
    for (int a = 0; a < N - 1; ++a) t.psi_dt[a] = static_cast<float>(s.psi[a] * dt);
    scal.resize(sizeof(t));
    std::memcpy(scal.data(), &t, sizeof(t));
}

template <int N>
cudaError_t launch_tc_t(const BlockArgs<float> &a, const std::vector<unsigned char> &scal, const void *bimg,
                        int sms, cudaStream_t st) {
    using S = TcShape<N>;
    if (a.tile + 2 * a.halo != S::ROWS || scal.size() != sizeof(TcScalars<N>)) return cudaErrorInvalidValue;
    TcScalars<N> k;
    std::memcpy(&k, scal.data(), sizeof(k));
    auto kern = mln_tc_kernel<N>;
    static bool attr_set = false;  // per instantiation; the attribute is per device function
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int64_t ntiles = (a.n_cells + a.tile - 1) / a.tile;
    const int64_t groups = (ntiles + S::G - 1) / S::G;
    const unsigned grid = static_cast<unsigned>(groups < sms ? groups : sms);
    kern<<<grid, S::G * S::ROWS, S::SMEM, st>>>(a, k, static_cast<const uint4 *>(bimg), ntiles);
    return cudaGetLastError();
}

}  // namespace

bool tc_supported(int N) { return N == 5 || N == 6; }

int tc_rows() { return TcShape<6>::ROWS; }

bool pack_tc(const Setup &s, double dt, std::vector<unsigned char> &img, std::vector<unsigned char> &scal) {
    switch (s.N) {
    case 5: pack_tc_t<5>(s, dt, img, scal); return true;
    case 6: pack_tc_t<6>(s, dt, img, scal); return true;
    default: return false;
    }
}

cudaError_t launch_tc(int N, const BlockArgs<float> &a, const std::vector<unsigned char> &scal, const void *bimg,
                      int sms, cudaStream_t st) {
    switch (N) {
    case 5: return launch_tc_t<5>(a, scal, bimg, sms, st);
    case 6: return launch_tc_t<6>(a, scal, bimg, sms, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int NC, int KC, bool TA, bool ISSUE = true>
cudaError_t tc_product_t(const float *A, const double *B, float *C, std::string &err) {
    constexpr int ABYTES = TA ? 0 : 128 * KC * 4, BBYTES = NC * KC * 4;
    constexpr int smem = 2 * BBYTES + 2 * ABYTES + 16;
    std::vector<unsigned char> img;
    append_image(img, NC, KC, [&](int r, int k) { return B[r * KC + k]; });
    float *dA = nullptr, *dC = nullptr;
    void *dB = nullptr;
    unsigned int *dflag = nullptr, hflag = 0;
    cudaError_t e = cudaMalloc(&dA, 128 * KC * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dB, img.size());
    if (e == cudaSuccess) e = cudaMalloc(&dC, 128 * NC * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dflag, 4);
    if (e == cudaSuccess) e = cudaMemset(dflag, 0, 4);
    if (e == cudaSuccess) e = cudaMemcpy(dA, A, 128 * KC * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, img.data(), img.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(mln_tc_product_kernel<NC, KC, TA, ISSUE>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) {
        mln_tc_product_kernel<NC, KC, TA, ISSUE><<<1, 128, smem>>>(dA, static_cast<const uint4 *>(dB), dC, dflag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(C, dC, 128 * NC * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&hflag, dflag, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && hflag) err = "tensor-core product: completion wait timed out";
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dC);
    cudaFree(dflag);
    return e;
}

cudaError_t tc_product(int nc, int kc, bool tmem_a, const float *A, const double *B, float *C, std::string &err) {
#define MLN_TCP(NN, KK)                                                                                  \
    if (nc == NN && kc == KK)                                                                            \
        return tmem_a ? tc_product_t<NN, KK, true>(A, B, C, err) : tc_product_t<NN, KK, false>(A, B, C, err);
    MLN_TCP(32, 40)
    MLN_TCP(48, 32)
    MLN_TCP(48, 40)
    MLN_TCP(32, 24)
    MLN_TCP(16, 8)
#undef MLN_TCP
    return cudaErrorInvalidValue;
}

cudaError_t tc_wait_selftest(std::string &err) {
    std::vector<float> A(128 * 8, 0.0f), C(128 * 16);
    std::vector<double> B(16 * 8, 0.0);
    return tc_product_t<16, 8, true, false>(A.data(), B.data(), C.data(), err);
}

int tc_smem_bytes(int N) {
    switch (N) {
    case 5: return TcShape<5>::SMEM;
    case 6: return TcShape<6>::SMEM;
    default: return 0;
    }
}

}  // namespace mln
