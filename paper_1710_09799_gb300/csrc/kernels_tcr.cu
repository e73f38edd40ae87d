// Tensor-core cell model of the rotated basis (MLN_FORM_ROTATED, FP32 state,
// N = 5 and 6). The state of a medium cell is z = T^T y, the merged form's
// state in the real eigenbasis T of U (Eqs. 25-26), and a step is
//   z'' = z + (R(phi) - I) z          plane rotations by phi = theta E^n dt (CUDA cores)
//   [z - z'' ; dP/dt] = [C1z, cz ; wz^T, cm] [z'' ; 1]   one dense product (tensor cores)
// with C1z = T^T (A0^2 - I) T, cz = T^T (A0 b + b), wz = T^T A0^T w and
// cm = w . b + c (Eqs. 17, 23): the two half-steps of the Liouville part that
// meet between two rotations are one affine map, which in this basis is one
// (D + 1) x (D + 1) product per cell and step.
//
// The product runs as tcgen05.mma kind::f16 over 128 cells at a time (the
// MMA's M), with FP32 accumulation in tensor memory. Each operand is split
// into FP16 high and low parts (x = hi + lo to about 2^-22 relative) and the
// product is summed as hi*hi + hi*lo + lo*hi: three MMAs per K block of 16.
// FP16's range is set by powers of two that change no bits: the state is held
// scaled by 2^13 inside the kernel (|z| <= |d| <= sqrt(2), so the scaled
// state stays below 2^14 < 65504), and each row of the constant matrix is
// scaled by its own power of two, undone on the accumulator.
//
// A CTA holds four independent tiles of 128 cells (one warpgroup each, K-cell
// halo on both sides, as in the other cell models' temporal blocking); the
// warpgroups synchronise only among themselves, so the tensor core works on
// one tile's product while the others rotate and update their fields. The
// CTA is persistent over the tiles; the constant operand is staged once by a
// bulk copy. The state rows z'' are written by their threads into tensor
// memory (tcgen05.st), where the MMA reads them as its A operand.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "setup.h"
#include "tc.cuh"
#include "tc_kernel.h"

namespace mln {

template <int N>
struct TcrShape {
    static constexpr int D = Dims<N>::D, Q = Dims<N>::Q, P = 2 * Q;
    static constexpr int KA = (D + 1 + 15) / 16 * 16;  // K: the state and the constant-1 column
    static constexpr int NB = (D + 1 + 15) / 16 * 16;  // MMA N: D increments and dP/dt
    static constexpr int LR = (D + 1 + 7) / 8 * 8;     // accumulator columns read back
    static constexpr int G = 4;                        // warpgroups (tiles) per CTA
    static constexpr int ROWS = 128;
    // tensor-memory columns of one group: A hi | A lo | accumulator
    static constexpr int A_HI = 0, A_LO = 32, ACC = 64, GCOLS = 128;
    static constexpr uint32_t TMEM_COLS = static_cast<uint32_t>(G * GCOLS);
    static constexpr int BB = NB * KA * 2;             // one FP16 image of the constant operand
    static constexpr int BIMG = 2 * BB;                // hi and lo
    static constexpr int OFF_E = (BIMG + 127) / 128 * 128;
    static constexpr int OFF_H = OFF_E + G * ROWS * 4;
    static constexpr int OFF_BAR = OFF_H + G * ROWS * 4;
    static constexpr int SMEM = OFF_BAR + 8 * (G + 1) + 16;
    static_assert(KA / 2 <= A_LO - A_HI && A_LO + KA / 2 <= ACC, "tensor-memory columns of A");
    static_assert(ACC + NB <= GCOLS, "tensor-memory columns of the accumulator");
    static_assert(LR <= NB, "read-back beyond the accumulator");
    static_assert(BIMG % 16 == 0, "bulk copy size");
};

// Scale of the state inside the kernel (an exact power of two).
constexpr float kTcrStateScale = 8192.0f;

template <int N>
struct TcrScalars {
    float psi_dt[N - 1];           // (m_a - m_{N-1}) dt / hbar: base angles per unit field
    float inv_row[Dims<N>::D + 1]; // 1 / (the power of two that scales each row of the constant operand)
};

namespace {

// x = hi + lo for a pair: hi is x rounded to FP16 (one packed conversion),
// read back as FP32; lo = x - hi is exact in FP32 and rounded to FP16 in turn,
// so hi + lo = x to about 2^-22 relative (|x| < 65504).
__device__ __forceinline__ void split_f16x2(float x0, float x1, uint32_t &hi, uint32_t &lo) {
    hi = tc::pack_f16x2(x0, x1);
    float h0, h1;
    asm("{\n\t.reg .f16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;\n\t}"
        : "=f"(h0), "=f"(h1)
        : "r"(hi));
    lo = tc::pack_f16x2(x0 - h0, x1 - h1);
}

// Stage this thread's row of A (v[0..n), then 1.0 at column n, zero-padded to
// KA columns) as FP16 hi and lo images in tensor memory (columns t_hi, t_lo of
// this thread's lane; two elements per 32-bit column).
template <int KA, int n>
__device__ __forceinline__ void stage_row_f16(uint32_t t_hi, uint32_t t_lo, const float *v) {
    static_assert(n + 1 <= KA && KA % 16 == 0, "row width");
#pragma unroll
    for (int c = 0; c < KA; c += 16) {
        uint32_t h[8], l[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k0 = c + 2 * e, k1 = k0 + 1;
            if (k0 > n) {  // padding: zero in both parts, no conversion
                h[e] = l[e] = 0u;
                continue;
            }
            const float x0 = k0 < n ? v[k0] : 1.0f;
            const float x1 = k1 < n ? v[k1] : (k1 == n ? 1.0f : 0.0f);
            split_f16x2(x0, x1, h[e], l[e]);
        }
        tc::st_x8(t_hi + c / 2, h);
        tc::st_x8(t_lo + c / 2, l);
    }
}

// D = A B^T over K = KA: hi*hi + hi*lo + lo*hi, A in tensor memory (two FP16
// per column), B images in shared memory (K-major, no swizzle) given by the
// descriptors of their first K block (block kb starts kb * 256 bytes later,
// i.e. 16 units further in the descriptor's address field). One thread.
template <int KA>
__device__ __forceinline__ void issue_f16(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint64_t db_hi, uint64_t db_lo,
                                          uint32_t idesc) {
#pragma unroll
    for (int kb = 0; kb < KA / 16; ++kb) tc::mma_f16_ts(d, a_hi + kb * 8, db_hi + 16 * kb, idesc, kb > 0 ? 1u : 0u);
#pragma unroll
    for (int kb = 0; kb < KA / 16; ++kb) tc::mma_f16_ts(d, a_hi + kb * 8, db_lo + 16 * kb, idesc, 1u);
#pragma unroll
    for (int kb = 0; kb < KA / 16; ++kb) tc::mma_f16_ts(d, a_lo + kb * 8, db_hi + 16 * kb, idesc, 1u);
}

template <int cols>
__device__ __forceinline__ void read_acc(uint32_t taddr, float (&v)[cols]) {
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
    mln_tcr_kernel(const __grid_constant__ BlockArgs<float> a, const __grid_constant__ TcrScalars<N> k,
                   const uint4 *__restrict__ bimg, int64_t ntiles) {
    using S = TcrShape<N>;
    constexpr int D = S::D, Q = S::Q, G = S::G, ROWS = S::ROWS;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, g = tid / ROWS, j = tid % ROWS, warp = tid / 32;
    float *sE = reinterpret_cast<float *>(smem + S::OFF_E) + g * ROWS;
    float *sH = reinterpret_cast<float *>(smem + S::OFF_H) + g * ROWS;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S::OFF_BAR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + S::OFF_BAR + 8 * (G + 1));

    // launched with a programmatic dependency on the kernel before it: wait
    // for that grid (its fields and states visible) before any global access
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    // the constant operand: one bulk copy into shared memory, completion on bars[G]
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
    const uint32_t tg = tmem + static_cast<uint32_t>(g * S::GCOLS);        // group's columns, lane 0
    const uint32_t lanes = static_cast<uint32_t>((warp % 4) * 32) << 16;  // this warp's lanes
    const uint32_t bar = tc::smem_addr(&bars[g]);
    const uint32_t a_hi = tg + S::A_HI, a_lo = tg + S::A_LO, acc = tg + S::ACC;
    const uint32_t b_hi = tc::smem_addr(smem), b_lo = b_hi + S::BB;
    const uint32_t idesc = tc::idesc_f16(S::NB);
    // descriptors of the constant operand's images (K-major, 8-row groups KA * 16 bytes apart)
    const uint64_t db_hi = tc::smem_desc(b_hi, 128, S::KA * 16), db_lo = tc::smem_desc(b_lo, 128, S::KA * 16);
    const int bar_id = 1 + g;
    const bool mma_warp = warp % 4 == 0;  // the group's first warp issues its MMAs
    uint32_t phase = 0;

    const int64_t n = a.n_cells;
    const bool periodic = a.boundary == 0;
    for (int64_t tile_index = static_cast<int64_t>(blockIdx.x) * G + g; tile_index < ntiles;
         tile_index += static_cast<int64_t>(gridDim.x) * G) {
        const int64_t t0 = tile_index * a.tile;
        const int64_t t1 = min(t0 + a.tile, n);
        // a tile that starts at the Mur cell loads one more cell on the left:
        // the Mur cell's value comes from its left neighbour's row in the same step
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
        float z[D];  // the state, scaled by kTcrStateScale
#pragma unroll
        for (int i = 0; i < D; ++i) z[i] = medium ? a.s_in[i * a.stride + m] * kTcrStateScale : 0.0f;
        float e = loaded ? a.E_in[gm] : 0.0f;
        float h = loaded ? a.H_in[gm] : 0.0f;
        sE[j] = e;
        sH[j] = h;
        const bool h_upd = loaded && (j + 1 < L) && (periodic || gm < n - 1);
        const bool e_upd = loaded && j >= 1 && (periodic || (gm > 0 && gm < n - 1));
        const bool mur = !periodic && loaded && gm == n - 2 && j + 1 < L;
        const bool is_src = a.src != nullptr && loaded && gm == a.source_cell;
        tc::bar_sync(bar_id, ROWS);

        for (int st = 0; st < a.nsteps; ++st) {
            if (h_upd) {
                h = fma(a.ch, sE[j + 1] - e, h);
                sH[j] = h;
            }
            // z'' = z + (R(phi) - I) z on the plane pairs, phi from E^n
            if (medium) {
                float sn[Q], c1[Q];
                plane_terms<N>(k.psi_dt, e, sn, c1);
#pragma unroll
                for (int p = 0; p < Q; ++p) {
                    const float x = z[2 * p], y = z[2 * p + 1];
                    z[2 * p] = x + fma(c1[p], x, sn[p] * y);
                    z[2 * p + 1] = y + fma(c1[p], y, -(sn[p] * x));
                }
            }
            stage_row_f16<S::KA, D>(a_hi + lanes, a_lo + lanes, z);
            tc::st_wait();
            tc::fence_before_sync();
            tc::bar_sync(bar_id, ROWS);  // A staged, H^{n+1/2} published
            // one elected lane of the group's first warp issues, from a converged
            // warp: about three times faster than issuing from a branch on the lane
            if (mma_warp) {
                if (tc::elect_one()) {
                    tc::fence_after_sync();
                    issue_f16<S::KA>(acc, a_hi, a_lo, db_hi, db_lo, idesc);
                    tc::mma_commit(bar);
                }
                __syncwarp();
            }
            // one MMA round trip is a few hundred cycles: suspend rather than spin
            // (at most 2^15 polls of 100 us each)
            ok = tc::mbar_wait_hint(bar, phase, 100000u, 1 << 15) && ok;
            phase ^= 1;
            tc::fence_after_sync();
            float v[S::LR];
            read_acc<S::LR>(acc + lanes, v);
            tc::ld_wait();
            float dpdt = 0.0f;
            if (medium) {
#pragma unroll
                for (int i = 0; i < D; ++i) z[i] = fma(v[i], k.inv_row[i], z[i]);
                dpdt = v[D] * k.inv_row[D];
            }
            float en = e;
            if (e_upd) en = fma(a.ca, e, a.cb * fma(h - sH[j - 1], a.inv_dx, -dpdt));
            float e_mur = 0.0f;
            if (mur) e_mur = fma(a.kappa, en - sE[j + 1], e);
            if (is_src) {
                const float s = static_cast<float>(a.src[st]);
                en = (a.source_kind == 1) ? s : en + s;
            }
            if (mur) {
                if (a.src != nullptr && a.source_cell == n - 1) {
                    const float s = static_cast<float>(a.src[st]);
                    e_mur = (a.source_kind == 1) ? s : e_mur + s;
                }
                sE[j + 1] = e_mur;
            }
            e = en;
            if (loaded && !(!periodic && gm == n - 1)) sE[j] = e;
            tc::fence_before_sync();
            tc::bar_sync(bar_id, ROWS);  // E^{n+1} published; the accumulator read by every row
            if (!periodic && loaded && gm == n - 1) e = sE[j];
        }

        const bool interior = loaded && j >= lh && j < lh + static_cast<int>(t1 - t0);
        if (interior) {
            a.E_out[gm] = e;
            a.H_out[gm] = h;
            if (medium) {
#pragma unroll
                for (int i = 0; i < D; ++i) a.s_out[i * a.stride + m] = z[i] * (1.0f / kTcrStateScale);
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
// Diagnostic product C = A B^T (A: 128 x KC floats, B: NC x KC, given in FP64)
// through the same scaling, split, staging and issue path as the step kernel:
// A scaled by `ascale` and split on the device, B's rows scaled by powers of
// two and split on the host, the scales undone on the accumulator. K = KC
// columns of A are staged as given (no constant column).
template <int NC, int KC>
__global__ void __launch_bounds__(128, 1)
    mln_tcr_product_kernel(const float *__restrict__ A, float ascale, const uint4 *__restrict__ bimg,
                           const float *__restrict__ inv_row, float *__restrict__ C, unsigned int *flag) {
    constexpr int BB = NC * KC * 2;
    constexpr uint32_t COLS = 256;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * BB);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    const int j = threadIdx.x, warp = j / 32;
    for (int o = j; o < 2 * BB / 16; o += 128) reinterpret_cast<uint4 *>(smem)[o] = bimg[o];
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
    const uint32_t acc = tmem + 128;
#pragma unroll
    for (int c = 0; c < KC; c += 16) {
        uint32_t h[8], l[8];
#pragma unroll
        for (int e = 0; e < 8; ++e)
            split_f16x2(A[j * KC + c + 2 * e] * ascale, A[j * KC + c + 2 * e + 1] * ascale, h[e], l[e]);
        tc::st_x8(tmem + lane + c / 2, h);
        tc::st_x8(tmem + lane + 64 + c / 2, l);
    }
    tc::st_wait();
    tc::fence_before_sync();
    __syncthreads();
    if (j == 0) {
        tc::fence_after_sync();
        const uint32_t bh = tc::smem_addr(smem);
        issue_f16<KC>(acc, tmem, tmem + 64, tc::smem_desc(bh, 128, KC * 16), tc::smem_desc(bh + BB, 128, KC * 16),
                      tc::idesc_f16(NC));
        tc::mma_commit(tc::smem_addr(bar));
    }
    const bool ok = tc::mbar_wait(tc::smem_addr(bar), 0);
    tc::fence_after_sync();
    float c[NC];
    read_acc<NC>(acc + lane, c);
    tc::ld_wait();
#pragma unroll
    for (int i = 0; i < NC; ++i) C[j * NC + i] = c[i] * inv_row[i] * (1.0f / ascale);
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

uint16_t f16_bits(float f) {
    // round to nearest even, FP16 normal and subnormal range (|f| < 65520)
    uint32_t b;
    std::memcpy(&b, &f, 4);
    const uint32_t sign = (b >> 16) & 0x8000u;
    const float a = std::fabs(f);
    if (a == 0.0f) return static_cast<uint16_t>(sign);
    int ex;
    std::frexp(a, &ex);  // a = m 2^ex, m in [0.5, 1)
    // spacing of FP16 values near a: 2^(ex - 11) for normals, 2^-24 for subnormals
    const int q = std::max(ex - 11, -24);
    const float u = std::nearbyint(std::ldexp(a, -q));  // round half to even (default rounding mode)
    const double v = std::ldexp(static_cast<double>(u), q);
    if (v == 0.0) return static_cast<uint16_t>(sign);  // below half the smallest subnormal
    // encode v = (1 + f/1024) 2^E or f 2^-24
    int e2;
    const double mv = std::frexp(v, &e2);  // v = mv 2^e2, mv in [0.5, 1)
    const int E = e2 - 1;
    if (E < -14) return static_cast<uint16_t>(sign | static_cast<uint32_t>(std::ldexp(v, 24)));
    const uint32_t frac = static_cast<uint32_t>(std::ldexp(mv * 2.0 - 1.0, 10));
    return static_cast<uint16_t>(sign | (static_cast<uint32_t>(E + 15) << 10) | frac);
}

float f16_value(uint16_t h) {
    const int e = (h >> 10) & 0x1F, f = h & 0x3FF;
    const float v = e == 0 ? std::ldexp(static_cast<float>(f), -24) : std::ldexp(1.0f + f / 1024.0f, e - 15);
    return (h & 0x8000u) ? -v : v;
}

// Power of two that brings a row's largest magnitude into (2^12, 2^13]
// (1 for a zero row).
double row_scale(const double *row, int n) {
    double mx = 0.0;
    for (int i = 0; i < n; ++i) mx = std::max(mx, std::fabs(row[i]));
    if (mx == 0.0 || !std::isfinite(mx)) return 1.0;
    int ex;
    std::frexp(mx, &ex);  // mx in [2^(ex-1), 2^ex)
    return std::ldexp(1.0, 13 - ex);
}

// FP16 hi and lo images (K-major core-matrix layout) of an R x K operand whose
// rows are already scaled: entry (r, k) = f(r, k), appended to out.
template <typename F>
void append_image16(std::vector<unsigned char> &out, int R, int K, F f) {
    std::vector<unsigned char> hi(static_cast<size_t>(R) * K * 2, 0), lo(hi.size(), 0);
    for (int r = 0; r < R; ++r)
        for (int k = 0; k < K; ++k) {
            const double x = f(r, k);
            const uint16_t h = f16_bits(static_cast<float>(x));
            const uint16_t l = f16_bits(static_cast<float>(x - static_cast<double>(f16_value(h))));
            std::memcpy(hi.data() + tc::core_offset16(r, k, K), &h, 2);
            std::memcpy(lo.data() + tc::core_offset16(r, k, K), &l, 2);
        }
    out.insert(out.end(), hi.begin(), hi.end());
    out.insert(out.end(), lo.begin(), lo.end());
}

template <int N>
void pack_tcr_t(const Setup &s, double dt, std::vector<unsigned char> &img, std::vector<unsigned char> &scal) {
    using S = TcrShape<N>;
    constexpr int D = S::D;
    // rows i < D: [C1z_i | 2^13 cz_i] (the state is scaled by 2^13, the
    // constant column carries 1); row D: [2^-13 wz | cm]
    std::vector<double> B(static_cast<size_t>(D + 1) * (D + 1));
    const double sc = static_cast<double>(kTcrStateScale);
    for (int i = 0; i < D; ++i) {
        for (int k = 0; k < D; ++k) B[i * (D + 1) + k] = s.C1z[i * D + k];
        B[i * (D + 1) + D] = sc * s.cz[i];
    }
    for (int k = 0; k < D; ++k) B[D * (D + 1) + k] = s.wz[k] / sc;
    B[D * (D + 1) + D] = s.cm;
    TcrScalars<N> t;
    std::memset(&t, 0, sizeof(t));
    std::vector<double> rs(D + 1);
    for (int i = 0; i <= D; ++i) {
        rs[i] = row_scale(&B[i * (D + 1)], D + 1);
        t.inv_row[i] = static_cast<float>(1.0 / rs[i]);
    }
    for (int a = 0; a < N - 1; ++a) t.psi_dt[a] = static_cast<float>(s.psi[a] * dt);
    img.clear();
    append_image16(img, S::NB, S::KA, [&](int r, int k) {
        return (r <= D && k <= D) ? rs[r] * B[r * (D + 1) + k] : 0.0;
    });
    scal.resize(sizeof(t));
    std::memcpy(scal.data(), &t, sizeof(t));
}

template <int N>
cudaError_t launch_tcr_t(const BlockArgs<float> &a, const std::vector<unsigned char> &scal, const void *bimg,
                         int sms, cudaStream_t st) {
    using S = TcrShape<N>;
    if (a.tile + 2 * a.halo != S::ROWS || scal.size() != sizeof(TcrScalars<N>)) return cudaErrorInvalidValue;
    TcrScalars<N> k;
    std::memcpy(&k, scal.data(), sizeof(k));
    auto kern = mln_tcr_kernel<N>;
    static bool attr_set = false;  // per instantiation; the attribute is per device function
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int64_t ntiles = (a.n_cells + a.tile - 1) / a.tile;
    const int64_t groups = (ntiles + S::G - 1) / S::G;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(static_cast<unsigned>(groups < sms ? groups : sms));
    cfg.blockDim = dim3(S::G * S::ROWS);
    cfg.dynamicSmemBytes = S::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a, k, static_cast<const uint4 *>(bimg), ntiles);
}

template <int NC, int KC>
cudaError_t tcr_product_t(const float *A, const double *B, float *C, std::string &err) {
    constexpr int BB = NC * KC * 2, smem = 2 * BB + 16;
    std::vector<double> rs(NC);
    std::vector<float> inv(NC);
    for (int r = 0; r < NC; ++r) {
        rs[r] = row_scale(B + r * KC, KC);
        inv[r] = static_cast<float>(1.0 / rs[r]);
    }
    std::vector<unsigned char> img;
    append_image16(img, NC, KC, [&](int r, int k) { return rs[r] * B[r * KC + k]; });
    float amax = 0.0f;
    for (int i = 0; i < 128 * KC; ++i) amax = std::max(amax, std::fabs(A[i]));
    int ex = 0;
    if (amax > 0.0f) std::frexp(amax, &ex);
    const float ascale = std::ldexp(1.0f, 13 - ex);
    float *dA = nullptr, *dC = nullptr, *dInv = nullptr;
    void *dB = nullptr;
    unsigned int *dflag = nullptr, hflag = 0;
    cudaError_t e = cudaMalloc(&dA, 128 * KC * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dB, img.size());
    if (e == cudaSuccess) e = cudaMalloc(&dC, 128 * NC * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dInv, NC * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dflag, 4);
    if (e == cudaSuccess) e = cudaMemset(dflag, 0, 4);
    if (e == cudaSuccess) e = cudaMemcpy(dA, A, 128 * KC * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, img.data(), img.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dInv, inv.data(), NC * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mln_tcr_product_kernel<NC, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) {
        mln_tcr_product_kernel<NC, KC><<<1, 128, smem>>>(dA, ascale, static_cast<const uint4 *>(dB), dInv, dC, dflag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(C, dC, 128 * NC * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&hflag, dflag, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && hflag) err = "tensor-core product: completion wait timed out";
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dC);
    cudaFree(dInv);
    cudaFree(dflag);
    return e;
}

}  // namespace

bool pack_tcr(const Setup &s, double dt, std::vector<unsigned char> &img, std::vector<unsigned char> &scal) {
    switch (s.N) {
    case 5: pack_tcr_t<5>(s, dt, img, scal); return true;
    case 6: pack_tcr_t<6>(s, dt, img, scal); return true;
    default: return false;
    }
}

cudaError_t launch_tcr(int N, const BlockArgs<float> &a, const std::vector<unsigned char> &scal, const void *bimg,
                       int sms, cudaStream_t st) {
    switch (N) {
    case 5: return launch_tcr_t<5>(a, scal, bimg, sms, st);
    case 6: return launch_tcr_t<6>(a, scal, bimg, sms, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t tcr_product(int nc, int kc, const float *A, const double *B, float *C, std::string &err) {
    if (nc == 48 && kc == 48) return tcr_product_t<48, 48>(A, B, C, err);
    if (nc == 32 && kc == 32) return tcr_product_t<32, 32>(A, B, C, err);
    if (nc == 16 && kc == 16) return tcr_product_t<16, 16>(A, B, C, err);
    return cudaErrorInvalidValue;
}

int tcr_smem_bytes(int N) {
    switch (N) {
    case 5: return TcrShape<5>::SMEM;
    case 6: return TcrShape<6>::SMEM;
    default: return 0;
    }
}

}  // namespace mln
