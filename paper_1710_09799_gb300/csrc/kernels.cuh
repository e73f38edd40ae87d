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

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <stdint.h>
#endif

namespace mln {

template <int N>
struct Dims {
    static constexpr int D = N * N - 1;      // adjoint dimension
    static constexpr int Q = N * (N - 1) / 2; // rotation planes of U
};

// Every propagator is applied as identity + increment: a cell's adjoint vector
// holds O(1) population components next to small coherences, and a product
// with a near-identity matrix would otherwise round the coherences at the
// scale of the populations in every step.
//
// Literal form (Eq. 23 with the diagonalisation of Eqs. 25-26), per step:
//   d'  = d  + (Dl d  + b)            Dl = A0 - I, A0 = exp(M dt/2)     (23a)
//   z   = T^T d'                      coordinates in the eigenbasis of U
//   d'' = d' + T (R(E) - I) z         R: plane rotations by theta_k E dt (23b, 25)
//   d   = d'' + (Dl d'' + b)                                             (23c)
//   dP/dt = w . d + c                                                    (Eq. 17)
template <int N, typename R>
struct StrangConsts {
    R Dl[Dims<N>::D * Dims<N>::D];
    R T[Dims<N>::D * Dims<N>::D];
    R b[Dims<N>::D];
    R w[Dims<N>::D];
    R psi_dt[N - 1];
    R c;
};

// Merged form: the second half-step of step n and the first of step n+1 are
// one affine map A0^2 y + (A0 b + b). The state is y = d' (after the first
// half-step); per step:
//   z = T^T y;  y'' = y + T (R(E) - I) z;
//   dP/dt = wm . y'' + cm              wm = A0^T w, cm = w . b + c  (= w . (A0 y'' + b) + c)
//   y = y'' + (C1 y'' + b2)            C1 = A0^2 - I, b2 = A0 b + b
template <int N, typename R>
struct MergedConsts {
    R C1[Dims<N>::D * Dims<N>::D];
    R T[Dims<N>::D * Dims<N>::D];
    R b2[Dims<N>::D];
    R wm[Dims<N>::D];
    R psi_dt[N - 1];
    R cm;
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
    // optional record of every step (nullptr: none): after step st the
    // interior cells also write E, H and the state to rec_E, rec_H, rec_S
    // advanced by st * rec_set bytes (the adjoint's recomputed segment);
    // a cell model that traces its intermediates (StrangTraceCell) writes
    // those of step st to rec_I advanced by st * rec_set bytes
    R *rec_E, *rec_H, *rec_S;
    int64_t rec_set;
    R *rec_I;
    // mln_trace_kernel only: launches with gridDim.y > 1 run independent
    // segments side by side, segment y with every buffer pointer advanced by
    // y * seg_bytes bytes and src by y * seg_src samples
    int64_t seg_bytes, seg_src;
    int64_t n_cells, mb, me, stride, source_cell;
    int32_t nsteps, halo, tile, boundary, source_kind, pad_;
    R ch, ca, cb, inv_dx, kappa;
};

__device__ __forceinline__ void sincos_r(double x, double *s, double *c) { sincos(x, s, c); }
__device__ __forceinline__ void sincos_r(float x, float *s, float *c) { sincosf(x, s, c); }

// Truncated Taylor series of sin x and cos x - 1 for |x| <= 1/8, bounded by
// the Lagrange remainder: FP64 up to x^11 / x^12 (remainder below
// 2^-36/13! ~ 2e-21 relative), fewer terms for smaller |x|; FP32 up to
// x^7 / x^8 (remainder below 2^-24/9! ~ 2e-13).
template <typename R>
struct SmallAngle;
template <>
struct SmallAngle<double> {
    static constexpr double kMax = 0.125;
    // Three tiers by |x|: the number of terms is the fewest that keeps the
    // remainder below 1e-20 relative (|x| <= 2^-16: to x^3 / x^4;
    // |x| <= 2^-6: to x^7 / x^8; |x| <= 1/8: to x^11 / x^12).
    __device__ __forceinline__ static void eval(double x, double &s, double &c1) {
        const double x2 = x * x;
        const double ax = fabs(x);
        if (ax <= 0x1p-16) {
            s = fma(x * x2, -1.0 / 6.0, x);
            c1 = x2 * fma(x2, 1.0 / 24.0, -0.5);
        } else if (ax <= 0x1p-6) {
            double ps = fma(x2, -1.0 / 5040.0, 1.0 / 120.0);
            ps = fma(ps, x2, -1.0 / 6.0);
            s = fma(x * x2, ps, x);
            double pc = fma(x2, 1.0 / 40320.0, -1.0 / 720.0);
            pc = fma(pc, x2, 1.0 / 24.0);
            pc = fma(pc, x2, -0.5);
            c1 = x2 * pc;
        } else {
            double ps = -1.0 / 39916800.0;                 // -1/11!
            ps = fma(ps, x2, 1.0 / 362880.0);              //  1/9!
            ps = fma(ps, x2, -1.0 / 5040.0);               // -1/7!
            ps = fma(ps, x2, 1.0 / 120.0);                 //  1/5!
            ps = fma(ps, x2, -1.0 / 6.0);                  // -1/3!
            s = fma(x * x2, ps, x);
            double pc = 1.0 / 479001600.0;                 //  1/12!
            pc = fma(pc, x2, -1.0 / 3628800.0);            // -1/10!
            pc = fma(pc, x2, 1.0 / 40320.0);               //  1/8!
            pc = fma(pc, x2, -1.0 / 720.0);                // -1/6!
            pc = fma(pc, x2, 1.0 / 24.0);                  //  1/4!
            pc = fma(pc, x2, -0.5);                        // -1/2!
            c1 = x2 * pc;
        }
    }
};
template <>
struct SmallAngle<float> {
    static constexpr float kMax = 0.125f;
    __device__ __forceinline__ static void eval(float x, float &s, float &c1) {
        const float x2 = x * x;
        float ps = -1.0f / 5040.0f;
        ps = fmaf(ps, x2, 1.0f / 120.0f);
        ps = fmaf(ps, x2, -1.0f / 6.0f);
        s = fmaf(x * x2, ps, x);
        float pc = 1.0f / 40320.0f;
        pc = fmaf(pc, x2, -1.0f / 720.0f);
        pc = fmaf(pc, x2, 1.0f / 24.0f);
        pc = fmaf(pc, x2, -0.5f);
        c1 = x2 * pc;
    }
};

// (sin x, cos x - 1) without cancellation: the series for small |x|, else
// sin x = 2 sin(x/2) cos(x/2) and cos x - 1 = -2 sin^2(x/2) from the library.
template <typename R>
__device__ __forceinline__ void sin_cosm1(R x, R &s, R &c1) {
    if (fabs(x) <= SmallAngle<R>::kMax) {
        SmallAngle<R>::eval(x, s, c1);
    } else {
        R sh, ch;
        sincos_r(x * R(0.5), &sh, &ch);
        s = R(2) * sh * ch;
        c1 = R(-2) * sh * sh;
    }
}

// (sin phi_k, cos phi_k - 1) for the q planes of T. Plane (a, b), a < b, in
// row-major pair order turns by phi_ab = (m_a - m_b) E dt / hbar (m: the
// eigenvalues of mu). Only the N-1 angles psi_a = (m_a - m_{N-1}) E dt / hbar
// are evaluated; phi_ab = psi_a - psi_b follows by the subtraction formulas
// written for (sin, cos - 1):
//   sin(p - r)     = s_p - s_r + s_p c1_r - c1_p s_r
//   cos(p - r) - 1 = c1_p + c1_r + c1_p c1_r + s_p s_r
template <int N, typename R>
__device__ __forceinline__ void plane_terms(const R *psi_dt, R e, R (&s)[Dims<N>::Q], R (&c1)[Dims<N>::Q]) {
    R sp[N], cp[N];
#pragma unroll
    for (int a = 0; a < N - 1; ++a) sin_cosm1(psi_dt[a] * e, sp[a], cp[a]);
    sp[N - 1] = R(0);
    cp[N - 1] = R(0);
    int k = 0;
#pragma unroll
    for (int a = 0; a < N; ++a) {
#pragma unroll
        for (int b = a + 1; b < N; ++b) {
            if (b == N - 1) {
                s[k] = sp[a];
                c1[k] = cp[a];
            } else {  // three operations each: the two products fused onto the sum
                s[k] = fma(sp[a], cp[b], fma(-cp[a], sp[b], sp[a] - sp[b]));
                c1[k] = fma(cp[a], cp[b], fma(sp[a], sp[b], cp[a] + cp[b]));
            }
            ++k;
        }
    }
}

// z <- (R(E) - I) z for the q planes of T: plane k turns (x, y) to
// (x cos phi + y sin phi, -x sin phi + y cos phi), the flow of the block
// [[0, theta], [-theta, 0]] of T^T U T over E dt; the null space of U (the
// last N - 1 coordinates) does not change.
template <int N, typename R>
__device__ __forceinline__ void rotation_apply(R (&z)[Dims<N>::D], const R (&s)[Dims<N>::Q],
                                               const R (&c1)[Dims<N>::Q]) {
#pragma unroll
    for (int k = 0; k < Dims<N>::Q; ++k) {
        const R x = z[2 * k], y = z[2 * k + 1];
        z[2 * k] = fma(c1[k], x, s[k] * y);
        z[2 * k + 1] = fma(c1[k], y, -(s[k] * x));
    }
#pragma unroll
    for (int i = 2 * Dims<N>::Q; i < Dims<N>::D; ++i) z[i] = R(0);
}
template <int N, typename R>
__device__ __forceinline__ void rotation_increment(R (&z)[Dims<N>::D], const R *psi_dt, R e) {
    R s[Dims<N>::Q], c1[Dims<N>::Q];
    plane_terms<N>(psi_dt, e, s, c1);
    rotation_apply<N>(z, s, c1);
}

// ---------------------------------------------------------------------------
// Double-float arithmetic (the step of MLN_KERNEL_DF32): a value is the
// unevaluated sum h + l of two FP32 numbers with |l| <= ulp(h) / 2, about 48
// significant bits. An FP64 instruction holds its SM sub-partition's FP64
// pipe 64 times as long as an FP32 instruction holds the FP32 pipe (whatever
// the number of active lanes), so the step runs faster as FP32 pairs than in
// FP64, at 2^-48 instead of 2^-53 per operation. The error-free transformations are
// Knuth's two-sum and the product error from a fused multiply-add; the _rn
// intrinsics keep the compiler from contracting any of their operations.
struct Df {
    float h, l;
};

__device__ __forceinline__ Df df_of(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - static_cast<double>(h))};  // x - h is exact in FP64
}
__device__ __forceinline__ double df_value(Df a) { return static_cast<double>(a.h) + static_cast<double>(a.l); }

// s + e = a + b exactly
__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// the pair (ah, al) as a normalised value
__device__ __forceinline__ Df df_norm(float ah, float al) {
    Df r;
    df_two_sum(ah, al, r.h, r.l);
    return r;
}
// (ah, al) = c x for c = ch + cl: the product's high part and, in the low
// word, its rounding error and the cross terms
__device__ __forceinline__ void df_first(float &ah, float &al, float ch, float cl, Df x) {
    ah = __fmul_rn(ch, x.h);
    al = __fmaf_rn(cl, x.h, __fmaf_rn(ch, x.l, __fmaf_rn(ch, x.h, -ah)));
}
__device__ __forceinline__ void df_first1(float &ah, float &al, float ch, Df x) {  // cl = 0
    ah = __fmul_rn(ch, x.h);
    al = __fmaf_rn(ch, x.l, __fmaf_rn(ch, x.h, -ah));
}
// (ah, al) += c x: the product's high part enters the high word exactly
// (two-sum), the errors of both the low word
__device__ __forceinline__ void df_acc(float &ah, float &al, float ch, float cl, Df x) {
    const float p = __fmul_rn(ch, x.h);
    const float pe = __fmaf_rn(cl, x.h, __fmaf_rn(ch, x.l, __fmaf_rn(ch, x.h, -p)));
    float s, e;
    df_two_sum(ah, p, s, e);
    ah = s;
    al = __fadd_rn(al, __fadd_rn(pe, e));
}
__device__ __forceinline__ void df_acc1(float &ah, float &al, float ch, Df x) {  // cl = 0
    const float p = __fmul_rn(ch, x.h);
    const float pe = __fmaf_rn(ch, x.l, __fmaf_rn(ch, x.h, -p));
    float s, e;
    df_two_sum(ah, p, s, e);
    ah = s;
    al = __fadd_rn(al, __fadd_rn(pe, e));
}
// (ah, al) += b for b = bh + bl
__device__ __forceinline__ void df_add(float &ah, float &al, float bh, float bl) {
    float s, e;
    df_two_sum(ah, bh, s, e);
    ah = s;
    al = __fadd_rn(al, __fadd_rn(bl, e));
}

// (sin x, cos x - 1) in double-float. For |x| <= 2^-12 the leading terms x
// and -x^2/2 in double-float and the rest of each series (below 2^-24 of the
// leading term, so FP32 suffices) as one FP32 correction:
//   sin x - x        = x x^2 (-1/6 + x^2/120),        |x^7/7!| < 2^-90 |x|,
//   cos x - 1 + x^2/2 = x^4 (1/24 - x^2/720),          |x^8/8!| < 2^-111 x^2.
// Larger angles take the FP64 evaluation.
__device__ __forceinline__ void df_sin_cosm1(Df x, Df &s, Df &c1) {
    if (fabsf(x.h) <= 0x1p-12f) {
        float x2h, x2l;
        x2h = __fmul_rn(x.h, x.h);
        x2l = __fmaf_rn(__fmul_rn(2.0f, x.h), x.l, __fmaf_rn(x.h, x.h, -x2h));
        const float ts = __fmul_rn(__fmul_rn(x.h, x2h), __fmaf_rn(x2h, 1.0f / 120.0f, -1.0f / 6.0f));
        float ah = x.h, al = x.l;
        df_add(ah, al, ts, 0.0f);
        s = df_norm(ah, al);
        const float tc = __fmul_rn(__fmul_rn(x2h, x2h), __fmaf_rn(x2h, -1.0f / 720.0f, 1.0f / 24.0f));
        ah = -0.5f * x2h;  // exact
        al = -0.5f * x2l;
        df_add(ah, al, tc, 0.0f);
        c1 = df_norm(ah, al);
    } else {
        double sd, cd;
        sin_cosm1(df_value(x), sd, cd);
        s = df_of(sd);
        c1 = df_of(cd);
    }
}

// The plane rotation of the merged step, z <- (R(E) - I) z, in double-float:
// the angles psi_a E dt (psi_dt as (hi, lo) pairs), the subtraction formulas
// and the rotation as in plane_terms and rotation_apply.
template <int N>
__device__ __forceinline__ void df_rotation_increment(Df (&z)[Dims<N>::D], const float *psi_h, const float *psi_l,
                                                      Df e) {
    constexpr int Q = Dims<N>::Q;
    Df sp[N], cp[N];
#pragma unroll
    for (int a = 0; a < N - 1; ++a) {
        float ah, al;
        df_first(ah, al, psi_h[a], psi_l[a], e);
        df_sin_cosm1(df_norm(ah, al), sp[a], cp[a]);
    }
    sp[N - 1] = Df{0.0f, 0.0f};
    cp[N - 1] = Df{0.0f, 0.0f};
    Df s[Q], c1[Q];
    int k = 0;
#pragma unroll
    for (int a = 0; a < N; ++a) {
#pragma unroll
        for (int b = a + 1; b < N; ++b) {
            if (b == N - 1) {
                s[k] = sp[a];
                c1[k] = cp[a];
            } else {
                // sin(p - r) = s_p - s_r + s_p c1_r - c1_p s_r
                float ah = sp[a].h, al = sp[a].l;
                df_add(ah, al, -sp[b].h, -sp[b].l);
                df_acc(ah, al, -cp[a].h, -cp[a].l, sp[b]);
                df_acc(ah, al, sp[a].h, sp[a].l, cp[b]);
                s[k] = df_norm(ah, al);
                // cos(p - r) - 1 = c1_p + c1_r + c1_p c1_r + s_p s_r
                ah = cp[a].h;
                al = cp[a].l;
                df_add(ah, al, cp[b].h, cp[b].l);
                df_acc(ah, al, sp[a].h, sp[a].l, sp[b]);
                df_acc(ah, al, cp[a].h, cp[a].l, cp[b]);
                c1[k] = df_norm(ah, al);
            }
            ++k;
        }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const Df x = z[2 * q], y = z[2 * q + 1];
        float ah, al;
        df_first(ah, al, s[q].h, s[q].l, y);  // c1 x + s y
        df_acc(ah, al, c1[q].h, c1[q].l, x);
        z[2 * q] = df_norm(ah, al);
        df_first(ah, al, -s[q].h, -s[q].l, x);  // c1 y - s x
        df_acc(ah, al, c1[q].h, c1[q].l, y);
        z[2 * q + 1] = df_norm(ah, al);
    }
#pragma unroll
    for (int i = 2 * Q; i < Dims<N>::D; ++i) z[i] = Df{0.0f, 0.0f};
}

// y = x + (A x + b) with A row-major D x D held in the constant bank.
template <int D, typename R>
__device__ __forceinline__ void affine_inc(R (&y)[D], const R *A, const R (&x)[D], const R *b) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
        R acc = b[i];
#pragma unroll
        for (int j = 0; j < D; ++j) acc = fma(A[i * D + j], x[j], acc);
        y[i] = x[i] + acc;
    }
}

// y += A x
template <int D, typename R>
__device__ __forceinline__ void matvec_acc(R (&y)[D], const R *A, const R (&x)[D]) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
        R acc = A[i * D] * x[0];
#pragma unroll
        for (int j = 1; j < D; ++j) acc = fma(A[i * D + j], x[j], acc);
        y[i] = y[i] + acc;
    }
}

// y += A x accumulated onto y itself: every term a fused multiply-add, so
// each rounding is at the scale of the component it updates.
template <int D, typename R>
__device__ __forceinline__ void matvec_onto(R (&y)[D], const R *A, const R (&x)[D]) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
        R acc = y[i];
#pragma unroll
        for (int j = 0; j < D; ++j) acc = fma(A[i * D + j], x[j], acc);
        y[i] = acc;
    }
}

// z = (y + b) + A y, accumulated onto y + b.
template <int D, typename R>
__device__ __forceinline__ void affine_onto(R (&z)[D], const R *A, const R (&y)[D], const R *b) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
        R acc = y[i] + b[i];
#pragma unroll
        for (int j = 0; j < D; ++j) acc = fma(A[i * D + j], y[j], acc);
        z[i] = acc;
    }
}

// y = A^T x
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

// Generalised Rodrigues form (Eq. 27) of the interaction step, for N <= 4:
// exp(U E dt) = I + sum_k sin(a_k) S_k + (1 - cos a_k) S_k^2 with
// S_k = T Theta_k T^T and, in the orientation of this T, a_k = -phi_k, so
//   d'' = d' + sum_k (-sin(phi_k) S_k d' - (cos(phi_k) - 1) S_k^2 d').
// The rest of the step is the literal Strang form.
template <int N, typename R>
struct RodriguesConsts {
    R Dl[Dims<N>::D * Dims<N>::D];
    R S[Dims<N>::Q * Dims<N>::D * Dims<N>::D];
    R S2[Dims<N>::Q * Dims<N>::D * Dims<N>::D];
    R b[Dims<N>::D];
    R w[Dims<N>::D];
    R psi_dt[N - 1];
    R c;
};

// One Liouville step of one cell; returns dP/dt^{n+1/2}. Two D-vectors live.
template <int N, typename R>
__device__ __forceinline__ R cell_step(R (&s)[Dims<N>::D], R e, const StrangConsts<N, R> &k) {
    constexpr int D = Dims<N>::D;
    R y[D];
    affine_inc<D>(y, k.Dl, s, k.b);        // d' = A0 d + b
    matTvec<D>(s, k.T, y);                 // z = T^T d'
    rotation_increment<N>(s, k.psi_dt, e); // (R - I) z
    matvec_acc<D>(y, k.T, s);              // d'' = d' + T (R - I) z
    affine_inc<D>(s, k.Dl, y, k.b);        // d = A0 d'' + b
    return dot_bias<D>(k.w, s, k.c);
}

template <int N, typename R>
__device__ __forceinline__ R cell_step(R (&s)[Dims<N>::D], R e, const MergedConsts<N, R> &k) {
    constexpr int D = Dims<N>::D;
    R z[D];
    matTvec<D>(z, k.T, s);                 // z = T^T y
    rotation_increment<N>(z, k.psi_dt, e);
    // FP64 accumulates the increments onto the state (fewer operations; a few
    // extra roundings at the state's own scale); FP32 sums each increment
    // first, since a dense row's many roundings at the state's scale would show
    if constexpr (sizeof(R) == 8) matvec_onto<D>(s, k.T, z);  // y'' = y + T (R - I) z
    else matvec_acc<D>(s, k.T, z);
    const R dpdt = dot_bias<D>(k.wm, s, k.cm);
    if constexpr (sizeof(R) == 8) affine_onto<D>(z, k.C1, s, k.b2);  // y = (y'' + b2) + C1 y''
    else affine_inc<D>(z, k.C1, s, k.b2);                           // y = y'' + (C1 y'' + b2)
#pragma unroll
    for (int i = 0; i < D; ++i) s[i] = z[i];
    return dpdt;
}

template <int N, typename R>
__device__ __forceinline__ R cell_step(R (&s)[Dims<N>::D], R e, const RodriguesConsts<N, R> &k) {
    constexpr int D = Dims<N>::D, Q = Dims<N>::Q;
    R y[D];
    affine_inc<D>(y, k.Dl, s, k.b);  // d' = A0 d + b
    R sn[Q], c1[Q];
    plane_terms<N>(k.psi_dt, e, sn, c1);
#pragma unroll
    for (int i = 0; i < D; ++i) s[i] = R(0);  // accumulates the increment
#pragma unroll
    for (int p = 0; p < Q; ++p) {
        const R *Sp = k.S + p * D * D, *S2p = k.S2 + p * D * D;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            R u = Sp[i * D] * y[0], v = S2p[i * D] * y[0];
#pragma unroll
            for (int j = 1; j < D; ++j) {
                u = fma(Sp[i * D + j], y[j], u);
                v = fma(S2p[i * D + j], y[j], v);
            }
            s[i] = fma(-sn[p], u, fma(-c1[p], v, s[i]));
        }
    }
#pragma unroll
    for (int i = 0; i < D; ++i) y[i] = y[i] + s[i];  // d''
    affine_inc<D>(s, k.Dl, y, k.b);                  // d = A0 d'' + b
    return dot_bias<D>(k.w, s, k.c);
}

// Evaluates (sin x, cos x - 1) as the step kernels do (diagnostic entry point).
template <typename R>
__global__ void sin_cosm1_kernel(const double *x, int64_t n, double *s, double *c1) {
    int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    R sv, cv;
    sin_cosm1(static_cast<R>(x[i]), sv, cv);
    s[i] = sv;
    c1[i] = cv;
}

// Blocks have at most kMaxThreads threads, which leaves up to 128 registers per thread.
constexpr int kMaxThreads = 512;

// g mod n in [0, n) for a cell index of a periodic ring. Tiles and halos keep
// g within one ring length of [0, n), so one compare and add or subtract
// does it; a 64-bit remainder (a long instruction sequence on the FP64-poor
// pipes of this GPU) runs only for halos wider than the ring.
__host__ __device__ __forceinline__ int64_t wrap_index(int64_t g, int64_t n) {
    if (g < 0) g += n;
    else if (g >= n) g -= n;
    if (g < 0 || g >= n) {
        g %= n;
        if (g < 0) g += n;
    }
    return g;
}

// Shared memory of a block's field exchange: E and H, two buffers each.
template <typename R>
__host__ __device__ constexpr size_t field_smem(int threads) {
    return 4 * static_cast<size_t>(threads) * sizeof(R);
}

// Cell model with the medium state in registers and dense D x D products
// whose constants are kernel-parameter (constant-bank) operands (or, in the
// batched kernel, a structure in shared memory).
template <int N, typename R, typename K>
struct RegisterCell {
    static constexpr int D = Dims<N>::D;
    using Consts = K;
    R s[D];
    __device__ __forceinline__ void setup(unsigned char *, const K &) {}
    __device__ __forceinline__ void load(const R *src, int64_t stride, int64_t m) {
#pragma unroll
        for (int i = 0; i < D; ++i) s[i] = src[i * stride + m];
    }
    __device__ __forceinline__ void store(R *dst, int64_t stride, int64_t m) const {
#pragma unroll
        for (int i = 0; i < D; ++i) dst[i * stride + m] = s[i];
    }
    __device__ __forceinline__ R step(R e, const K &k) { return cell_step<N>(s, e, k); }
    __device__ __forceinline__ void end_step() {}
};

// p advanced by off bytes (nullptr stays nullptr).
template <typename T>
__device__ __forceinline__ T *byte_advance(T *p, int64_t off) {
    return p ? reinterpret_cast<T *>(reinterpret_cast<unsigned long long>(p) + static_cast<unsigned long long>(off))
             : p;
}

// Whether a cell model writes its intermediates (Cell::kTrace).
template <typename...>
using mln_void_t = void;
template <typename C, typename = void>
struct CellTraces {
    static constexpr bool value = false;
};
template <typename C>
struct CellTraces<C, mln_void_t<decltype(C::kTrace)>> {
    static constexpr bool value = C::kTrace;
};

// The Strang step of RegisterCell<N, R, StrangConsts> (same operations, same
// bits) that also writes the step's intermediates for the reverse sweep of
// the adjoint: rows 0..D-1 d' = A0 d + b, rows D..D+2q-1 the plane rows of
// z = T^T d', rows D+2q..2D+2q-1 d'' = d' + T (R - I) z, then (FP64) q rows
// of the planes' sin phi_k and q rows of cos phi_k - 1, each row `stride`
// apart, at the pointer given by trace_to before the step (nullptr: none).
template <int N, typename R>
struct StrangTraceCell {
    static constexpr int D = Dims<N>::D, P = 2 * Dims<N>::Q;
    static constexpr bool kTrace = true;
    using Consts = StrangConsts<N, R>;
    R s[D];
    R *tp = nullptr;
    int64_t ts = 0, tm = 0;
    __device__ __forceinline__ void setup(unsigned char *, const Consts &) {}
    __device__ __forceinline__ void load(const R *src, int64_t stride, int64_t m) {
#pragma unroll
        for (int i = 0; i < D; ++i) s[i] = src[i * stride + m];
    }
    __device__ __forceinline__ void store(R *dst, int64_t stride, int64_t m) const {
#pragma unroll
        for (int i = 0; i < D; ++i) dst[i * stride + m] = s[i];
    }
    __device__ __forceinline__ void trace_to(R *p, int64_t stride, int64_t m) {
        tp = p;
        ts = stride;
        tm = m;
    }
    __device__ __forceinline__ R step(R e, const Consts &k) {
        R y[D];
        affine_inc<D>(y, k.Dl, s, k.b);  // d' = A0 d + b
        if (tp) {
#pragma unroll
            for (int i = 0; i < D; ++i) tp[i * ts + tm] = y[i];
        }
        matTvec<D>(s, k.T, y);  // z = T^T d'
        if (tp) {
#pragma unroll
            for (int i = 0; i < P; ++i) tp[(D + i) * ts + tm] = s[i];
        }
        R sn[P / 2], c1[P / 2];
        plane_terms<N>(k.psi_dt, e, sn, c1);
        rotation_apply<N>(s, sn, c1);  // (R - I) z, as rotation_increment
        matvec_acc<D>(y, k.T, s);      // d'' = d' + T (R - I) z
        if (tp) {
#pragma unroll
            for (int i = 0; i < D; ++i) tp[(D + P + i) * ts + tm] = y[i];
            if constexpr (sizeof(R) == 8) {
#pragma unroll
                for (int i = 0; i < P / 2; ++i) {
                    tp[(2 * D + P + i) * ts + tm] = sn[i];
                    tp[(2 * D + P + P / 2 + i) * ts + tm] = c1[i];
                }
            }
        }
        affine_inc<D>(s, k.Dl, y, k.b);  // d = A0 d'' + b
        return dot_bias<D>(k.w, s, k.c);
    }
    __device__ __forceinline__ void end_step() {}
};

// Sparse program of the merged FP64 step: the non-zero entries of T^T
// (restricted to the 2q plane rows), T (restricted to the plane columns),
// A0^2 - I and A0^T w, row by row in ascending column order (the order of
// the dense products, so both give the same sums). Built once per context.
template <int N>
struct SparseConsts {
    double b2[Dims<N>::D];
    double psi_dt[N - 1];
    double cm;
    const int32_t *rowptr;  // entry index where each row starts, then the end of the last row:
                            // T^T rows 0..2q-1, T rows 2q.., C1 rows 2q+D.., wm row 2q+2D; 2q + 2D + 2 entries
    const int32_t *cols;    // column of each entry
    const double *vals;     // value of each entry
    int32_t nnz;            // entries in all four products
    int32_t nrowptr;        // length of rowptr
};

// Cell model with the medium state in shared memory (one column per thread)
// and products that walk the sparse program, also held in shared memory. On
// GB300 an FP64 FMA costs 16 issue slots' worth of FP64-pipe time per warp,
// so the extra shared-memory loads and loop control are free and only the
// non-zero entries cost time.
template <int N>
struct SharedSparseCell {
    static constexpr int D = Dims<N>::D, Q = Dims<N>::Q;
    using Consts = SparseConsts<N>;
    double *yc, *yn, *z;       // this thread's column: element i at [i * nt]
    const double *vals;
    const int32_t *offs, *rp;  // offs[e] = cols[e] * nt
    int nt;

    // Shared-memory bytes besides the E/H arrays.
    __host__ __device__ static size_t smem_bytes(int threads, int nnz, int nrowptr) {
        return static_cast<size_t>(threads) * (2 * D + 2 * Q) * sizeof(double) + static_cast<size_t>(nnz) * 12 +
               static_cast<size_t>(nrowptr) * 4;
    }

    // Block-cooperative: lay out the state columns and copy the program.
    __device__ __forceinline__ void setup(unsigned char *extra, const Consts &k) {
        nt = blockDim.x;
        const int t = threadIdx.x;
        double *base = reinterpret_cast<double *>(extra);
        yc = base + t;
        yn = base + D * nt + t;
        z = base + 2 * D * nt + t;
        double *v = base + (2 * D + 2 * Q) * nt;
        int32_t *o = reinterpret_cast<int32_t *>(v + k.nnz);
        int32_t *r = o + k.nnz;
        for (int e = t; e < k.nnz; e += nt) {
            v[e] = k.vals[e];
            o[e] = k.cols[e] * nt;
        }
        for (int e = t; e < k.nrowptr; e += nt) r[e] = k.rowptr[e];
        vals = v;
        offs = o;
        rp = r;
    }
    __device__ __forceinline__ void load(const double *src, int64_t stride, int64_t m) {
        for (int i = 0; i < D; ++i) yc[i * nt] = src[i * stride + m];
    }
    __device__ __forceinline__ void store(double *dst, int64_t stride, int64_t m) const {
        for (int i = 0; i < D; ++i) dst[i * stride + m] = yc[i * nt];
    }
    // sum over the entries of row r of a product with input column x
    __device__ __forceinline__ double row(int r, const double *x, double acc) const {
        const int e1 = rp[r + 1];
#pragma unroll 1
        for (int e = rp[r]; e < e1; ++e) acc = fma(vals[e], x[offs[e]], acc);
        return acc;
    }
    __device__ __forceinline__ double step(double e, const Consts &k) {
        // row bases in rowptr: T^T rows [0, 2q), T rows [2q, 2q + D), C1 rows
        // [2q + D, 2q + 2D), the wm row 2q + 2D; rowptr has 2q + 2D + 2 entries
        constexpr int rT = 2 * Q, rC = 2 * Q + D, rW = 2 * Q + 2 * D;
        // z = T^T y on the plane rows
#pragma unroll 1
        for (int r = 0; r < 2 * Q; ++r) z[r * nt] = row(r, yc, 0.0);
        // (R(E) - I) z
        double zz[D];
#pragma unroll
        for (int i = 0; i < 2 * Q; ++i) zz[i] = z[i * nt];
        rotation_increment<N>(zz, k.psi_dt, e);
#pragma unroll
        for (int i = 0; i < 2 * Q; ++i) z[i * nt] = zz[i];
        // y'' = y + T (R - I) z, accumulated onto y
#pragma unroll 1
        for (int r = 0; r < D; ++r) yc[r * nt] = row(rT + r, z, yc[r * nt]);
        const double dpdt = row(rW, yc, k.cm);
        // y = (y'' + b2) + C1 y'', accumulated onto y'' + b2 (no add where b2 is zero:
        // the same value as adding it)
#pragma unroll 1
        for (int r = 0; r < D; ++r) {
            const double b = k.b2[r];
            const double a0 = __double_as_longlong(b) != 0 ? yc[r * nt] + b : yc[r * nt];
            yn[r * nt] = row(rC + r, yc, a0);
        }
        return dpdt;
    }
    // every thread of the block swaps, medium or not, so the columns stay aligned
    __device__ __forceinline__ void end_step() {
        double *t = yc;
        yc = yn;
        yn = t;
    }
};

// Problem properties known when a kernel is compiled (the run-time compiled
// kernels know their grid): the code for the other cases is left out.
enum : unsigned {
    kBodyRing = 1u,   // every grid is a ring (no held cell, no Mur rule)
    kBodyOpen = 2u,   // every grid is open
    kBodyNoSrc = 4u,  // no source samples
    kBodyNoRec = 8u,  // no recording of the steps
    kBodyUnroll = 16u,  // two steps per loop iteration (buffers at fixed addresses; more registers)
    kBodyCg = 32u,      // inputs read through L2 only (ld.global.cg): other blocks of the same
                        // launch wrote them, and this SM's L1 may hold an older copy
};

// The type of E, H and dP/dt inside a block: R, or the cell model's own
// Field type (Df for the double-float model, whose field update then runs in
// pairs too, with no FP64 instruction per step).
template <typename C, typename R, typename = void>
struct CellField {
    using type = R;
};
template <typename C, typename R>
struct CellField<C, R, mln_void_t<typename C::Field>> {
    using type = typename C::Field;
};
// Values of type R in memory to and from the block's field type.
template <typename F, typename R>
struct FieldConv {
    __device__ __forceinline__ static F in(R v) { return v; }
    __device__ __forceinline__ static R out(F v) { return v; }
};
template <>
struct FieldConv<Df, double> {
    __device__ __forceinline__ static Df in(double v) { return df_of(v); }
    __device__ __forceinline__ static double out(Df v) { return df_value(v); }
};
// The field update's operations: for FP64 and FP32 the plain expressions
// (the same instructions as written out), for pairs their double-float forms.
template <typename F>
__device__ __forceinline__ F fld_sub(F a, F b) { return a - b; }
template <typename F>
__device__ __forceinline__ F fld_add(F a, F b) { return a + b; }
template <typename F>
__device__ __forceinline__ F fld_neg(F a) { return -a; }
template <typename F>
__device__ __forceinline__ F fld_mul(F c, F x) { return c * x; }
template <typename F>
__device__ __forceinline__ F fld_fma(F c, F x, F y) { return fma(c, x, y); }
template <typename F>
__device__ __forceinline__ bool fld_finite(F a) { return isfinite(a); }
template <>
__device__ __forceinline__ Df fld_sub(Df a, Df b) {
    float ah = a.h, al = a.l;
    df_add(ah, al, -b.h, -b.l);
    return df_norm(ah, al);
}
template <>
__device__ __forceinline__ Df fld_add(Df a, Df b) {
    float ah = a.h, al = a.l;
    df_add(ah, al, b.h, b.l);
    return df_norm(ah, al);
}
template <>
__device__ __forceinline__ Df fld_neg(Df a) { return Df{-a.h, -a.l}; }
template <>
__device__ __forceinline__ Df fld_mul(Df c, Df x) {
    float ah, al;
    df_first(ah, al, c.h, c.l, x);
    return df_norm(ah, al);
}
template <>
__device__ __forceinline__ Df fld_fma(Df c, Df x, Df y) {
    float ah = y.h, al = y.l;
    df_acc(ah, al, c.h, c.l, x);
    return df_norm(ah, al);
}
template <>
__device__ __forceinline__ bool fld_finite(Df a) { return isfinite(a.h) && isfinite(a.l); }

// One thread block advances tile `tile_index` of one grid by a.nsteps steps.
// smem: 2 * blockDim.x reals for E and H, then the cell model's extra space.
template <int N, typename R, typename Cell, unsigned kFlags = 0u>
__device__ __forceinline__ void block_body(const BlockArgs<R> &a, const typename Cell::Consts &k, int64_t tile_index,
                                           unsigned char *smem) {
    constexpr bool kRingOnly = (kFlags & kBodyRing) != 0, kOpenOnly = (kFlags & kBodyOpen) != 0;
    constexpr bool kNoSrc = (kFlags & kBodyNoSrc) != 0, kNoRec = (kFlags & kBodyNoRec) != 0;
    // E, H and dP/dt in the block: R, or the cell model's field type
    using F = typename CellField<Cell, R>::type;
    using Cv = FieldConv<F, R>;
    static_assert(sizeof(F) == sizeof(R), "the shared E and H buffers are sized for R");
    const F ch = Cv::in(a.ch), ca = Cv::in(a.ca), cb = Cv::in(a.cb), inv_dx = Cv::in(a.inv_dx);
    // E and H of the block, two buffers each: step st reads one and writes the other
    F *const bufE0 = reinterpret_cast<F *>(smem);
    F *const bufH0 = bufE0 + blockDim.x;
    F *const bufE1 = bufH0 + blockDim.x;
    F *const bufH1 = bufE1 + blockDim.x;

    const int j = threadIdx.x;
    const int64_t n = a.n_cells;
    const int64_t t0 = tile_index * a.tile;
    const int64_t t1 = min(t0 + a.tile, n);
    const bool periodic = kRingOnly ? true : (kOpenOnly ? false : a.boundary == 0);
    // The Mur cell's value comes from its left neighbour's thread in the same
    // step, so its dependence reaches one cell further left than a step's:
    // a tile that starts at the Mur cell loads one more cell on the left
    // (that tile has one cell, and a block of at least 2 halo + 1 threads,
    // rounded up to a warp, has a thread to spare).
    const int lh = a.halo + ((!periodic && t0 == n - 1) ? 1 : 0);
    const int L = static_cast<int>(t1 - t0) + lh + a.halo;
    const int64_t g = t0 - lh + j;
    int64_t gm = g;
    bool loaded = j < L;
    if (periodic) {
        gm = wrap_index(g, n);
    } else {
        loaded = loaded && g >= 0 && g < n;
    }
    const bool medium = loaded && gm >= a.mb && gm < a.me;
    const int64_t m = gm - a.mb;

    Cell cell;
    cell.setup(smem + field_smem<R>(blockDim.x), k);
    F e = F(), h = F();
    if constexpr ((kFlags & kBodyCg) != 0u) {
        if (loaded) {
            e = Cv::in(__ldcg(a.E_in + gm));
            h = Cv::in(__ldcg(a.H_in + gm));
        }
        if (medium) cell.load_cg(a.s_in, a.stride, m);
    } else {
        if (loaded) {
            e = Cv::in(a.E_in[gm]);
            h = Cv::in(a.H_in[gm]);
        }
        if (medium) cell.load(a.s_in, a.stride, m);
    }
    bufE0[j] = e;
    bufH0[j] = h;

    // H_{i+1/2} exists for every cell of a ring and for cells 0..n-2 of an open grid;
    // it needs E of the next loaded cell.
    const bool h_upd = loaded && (j + 1 < L) && (periodic || gm < n - 1);
    // E needs H_{i-1/2} of the previous loaded cell (whose H update always
    // exists then). On an open grid cell 0 is held (hard source only) and cell
    // n-1 is set by the Mur rule of cell n-2's thread.
    const bool e_upd = loaded && j >= 1 && (periodic || (gm > 0 && gm < n - 1));
    const bool mur = !periodic && loaded && gm == n - 2 && j + 1 < L;
    const bool mur_cell = !periodic && loaded && gm == n - 1;
    const bool has_src = !kNoSrc && a.src != nullptr;
    const bool is_src = has_src && loaded && gm == a.source_cell;
    const int tlen = static_cast<int>(t1 - t0);
    const bool interior = loaded && j >= lh && j < lh + tlen;
    const bool record = !kNoRec && a.rec_E != nullptr && interior;
    // Light cone: the tile's values after nsteps steps depend on the values
    // after step st only within nsteps - 1 - st cells of the tile; one cell
    // more keeps the Mur cell's left neighbour, whose thread computes the Mur
    // cell's value in the same step. A warp with no cell within
    // nsteps - st of the tile skips step st (and every later one: the region
    // only shrinks, so the values it leaves stale are never read).
    const int w0 = j & ~31;
    const int active = min(w0 + 32 - lh, lh + tlen - w0) + a.nsteps;  // steps this warp computes
    __syncthreads();

    // one step from buffers (cE, cH) into (nE, nH)
    auto step = [&](int st, const F *cE, const F *cH, F *nE, F *nH) {
        if (st < active) {  // warp-uniform
            if (h_upd) h = fld_fma(ch, fld_sub(cE[j + 1], e), h);
            // the previous cell's new H, with the operands and operations of its own thread
            F hl = F();
            if (e_upd) hl = fld_fma(ch, fld_sub(e, cE[j - 1]), cH[j - 1]);
            F dpdt = F();
            if constexpr (CellTraces<Cell>::value) {
                if (medium)
                    cell.trace_to(record ? reinterpret_cast<R *>(reinterpret_cast<char *>(a.rec_I) +
                                                                 static_cast<int64_t>(st) * a.rec_set)
                                         : nullptr,
                                  a.stride, m);
            }
            if (medium) dpdt = cell.step(e, k);
            cell.end_step();
            F en = e;
            if (e_upd) en = fld_fma(ca, e, fld_mul(cb, fld_fma(fld_sub(h, hl), inv_dx, fld_neg(dpdt))));
            F e_mur = F();
            if (mur) e_mur = fld_fma(Cv::in(a.kappa), fld_sub(en, cE[j + 1]), e);  // from E^{n+1} before any source
            if (is_src) {
                const F v = FieldConv<F, double>::in(a.src[st]);
                en = (a.source_kind == 1) ? v : fld_add(en, v);
            }
            if (mur) {
                if (has_src && a.source_cell == n - 1) {
                    const F v = FieldConv<F, double>::in(a.src[st]);
                    e_mur = (a.source_kind == 1) ? v : fld_add(e_mur, v);
                }
                nE[j + 1] = e_mur;
            }
            e = en;
            if (!mur_cell) nE[j] = e;
            nH[j] = h;
        }
        __syncthreads();
        // the Mur cell takes its new value from shared memory
        if (mur_cell) e = nE[j];
        if (record) {
            const int64_t off = static_cast<int64_t>(st) * a.rec_set;
            reinterpret_cast<R *>(reinterpret_cast<char *>(a.rec_E) + off)[gm] = Cv::out(e);
            reinterpret_cast<R *>(reinterpret_cast<char *>(a.rec_H) + off)[gm] = Cv::out(h);
            if (medium) cell.store(reinterpret_cast<R *>(reinterpret_cast<char *>(a.rec_S) + off), a.stride, m);
        }
    };
    if constexpr ((kFlags & kBodyUnroll) != 0u) {
        // two steps per iteration: the buffers alternate at fixed addresses
        int st = 0;
        for (; st + 1 < a.nsteps; st += 2) {
            step(st, bufE0, bufH0, bufE1, bufH1);
            step(st + 1, bufE1, bufH1, bufE0, bufH0);
        }
        if (st < a.nsteps) step(st, bufE0, bufH0, bufE1, bufH1);
    } else {
        F *cE = bufE0, *cH = bufH0, *nE = bufE1, *nH = bufH1;
        for (int st = 0; st < a.nsteps; ++st) {
            step(st, cE, cH, nE, nH);
            F *t = cE;
            cE = nE;
            nE = t;
            t = cH;
            cH = nH;
            nH = t;
        }
    }

    if (interior) {
        a.E_out[gm] = Cv::out(e);
        a.H_out[gm] = Cv::out(h);
        if (medium) cell.store(a.s_out, a.stride, m);
        if (!fld_finite(e)) atomicOr(a.flags, 1u);
    }
}

// ---------------------------------------------------------------------------
// Batches of independent grids: a table of grids and a work list of (grid,
// tile) items; one block per item.

// Shared-memory room for one grid's constants.
constexpr int kBatchConstsMax = 8192;
constexpr int kBatchMaxN = 4;
// Threads per block of the batched kernels (tile + 2 K <= this).
constexpr int kBatchThreads = 256;

template <typename R>
struct BatchGrid {
    R *E[2], *H[2], *S[2];   // buffer set 0 (caller's) and 1 (context's)
    const double *src;       // source samples from the batch's step 0, or nullptr
    unsigned int *flags;
    int64_t n_cells, mb, me, stride, source_cell;
    int32_t N, boundary, source_kind, consts_off, consts_bytes, pad_;
    R ch, ca, cb, inv_dx, kappa;
};

struct BatchItem {
    int32_t grid, tile;
};

// The block of one work item: stage the grid's constants (consts_bytes at
// consts + consts_off, a multiple of 16) at the start of shared memory, where
// the cell model reads them as its Consts, then run the fused steps.
template <int N, typename R, typename Cell, unsigned kFlags = 0u>
__device__ __forceinline__ void batch_body(const BatchGrid<R> *__restrict__ grids, const BatchItem *__restrict__ items,
                                           const unsigned char *__restrict__ consts, int parity, int nsteps,
                                           int halo, int tile, int64_t step_offset, unsigned char *smem_raw,
                                           int64_t item_index = -1) {
    const BatchItem it = items[item_index >= 0 ? item_index : static_cast<int64_t>(blockIdx.x)];
    const BatchGrid<R> &g = grids[it.grid];
    for (int o = threadIdx.x * 16; o < g.consts_bytes; o += blockDim.x * 16)
        *reinterpret_cast<uint4 *>(smem_raw + o) = *reinterpret_cast<const uint4 *>(consts + g.consts_off + o);
    __syncthreads();
    BlockArgs<R> a;
    a.E_in = g.E[parity];
    a.H_in = g.H[parity];
    a.s_in = g.S[parity];
    a.E_out = g.E[parity ^ 1];
    a.H_out = g.H[parity ^ 1];
    a.s_out = g.S[parity ^ 1];
    a.src = g.src ? g.src + step_offset : nullptr;
    a.flags = g.flags;
    a.rec_E = a.rec_H = a.rec_S = a.rec_I = nullptr;
    a.rec_set = 0;
    a.seg_bytes = a.seg_src = 0;
    a.n_cells = g.n_cells;
    a.mb = g.mb;
    a.me = g.me;
    a.stride = g.stride;
    a.source_cell = g.source_cell;
    a.nsteps = nsteps;
    a.halo = halo;
    a.tile = tile;
    a.boundary = g.boundary;
    a.source_kind = g.source_kind;
    a.pad_ = 0;
    a.ch = g.ch;
    a.ca = g.ca;
    a.cb = g.cb;
    a.inv_dx = g.inv_dx;
    a.kappa = g.kappa;
    block_body<N, R, Cell, kFlags>(a, *reinterpret_cast<const typename Cell::Consts *>(smem_raw), it.tile,
                           smem_raw + kBatchConstsMax);
}

// One persistent launch for all K-step chunks of a call over the work items
// of one N. Blocks take items (chunk c, item i) from a counter in
// chunk-major order; before chunk c of a tile, one thread waits until the
// tile and every tile of its grid within halo + 1 cells of it (those whose
// cells it reads, and whose reads cover its cells: the two neighbours, and a
// tile beyond a neighbour as short as the ragged last one) have completed
// chunk c - 1, then the block runs the chunk and publishes the tile's
// progress. An item is only taken by a block that is running, and it
// waits only for items with smaller indices, which running blocks hold, so
// the waits end without any guarantee of co-residency; each is still bounded
// (wait_limit polls; 0 gives up at once, for testing) and a wait that gives up
// sets bit 2 of the grid's flag word and lets the block go on.
struct BatchPersist {
    unsigned long long *work;  // next item index (zero at the launch)
    int *progress;             // chunks completed, per item of this N (zero at the launch)
    int64_t n_items;
    int32_t n_chunks, K, last_steps, wait_limit;
};

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until *progress >= c, for at most `limit` polls; false if it gave up.
__device__ __forceinline__ bool batch_wait(const int *progress, int c, int limit) {
    int polls = 0;
    while (ld_acquire(progress) < c) {
        if (++polls > limit) return false;
        __nanosleep(100);
    }
    return true;
}

// The waits before chunk c of item i (tile it.tile of its grid): the item
// itself, then outwards in each direction every tile of the grid whose cells
// start within halo + 1 cells of this tile (wrapping on a ring; the grid's
// tiles are consecutive items). False if a wait gave up.
template <typename R>
__device__ bool batch_wait_deps(const BatchGrid<R> &g, const BatchItem &it, const int *progress, int64_t i, int c,
                                int halo, int tile, int limit) {
    if (limit <= 0 || !batch_wait(progress + i, c, limit)) return false;
    const int64_t nt = (g.n_cells + tile - 1) / tile;
    for (int dir = -1; dir <= 1; dir += 2) {
        int64_t gap = 0;  // cells strictly between this tile and tile t
        for (int64_t s = 1; s < nt && gap <= halo; ++s) {
            int64_t t = it.tile + dir * s;
            if (t < 0 || t >= nt) {
                if (g.boundary != 0) break;  // open grid: nothing beyond its ends
                t = t < 0 ? t + nt : t - nt;
            }
            if (!batch_wait(progress + i + (t - it.tile), c, limit)) return false;
            gap += min(static_cast<int64_t>(tile), g.n_cells - t * tile);
        }
    }
    return true;
}

template <int N, typename R, typename Cell, unsigned kFlags = 0u>
__device__ __forceinline__ void batch_persistent(const BatchGrid<R> *__restrict__ grids,
                                                 const BatchItem *__restrict__ items,
                                                 const unsigned char *__restrict__ consts, int halo, int tile,
                                                 int64_t step_offset, const BatchPersist &p, unsigned char *smem_raw) {
    __shared__ long long q_sh;
    const int64_t total = static_cast<int64_t>(p.n_chunks) * p.n_items;
    for (;;) {
        if (threadIdx.x == 0) q_sh = static_cast<long long>(atomicAdd(p.work, 1ull));
        __syncthreads();
        const int64_t q = q_sh;
        __syncthreads();  // every thread has read q_sh before the next item's fetch
        if (q >= total) break;
        const int c = static_cast<int>(q / p.n_items);
        const int64_t i = q % p.n_items;
        if (threadIdx.x == 0 && c > 0) {
            const BatchItem it = items[i];
            if (!batch_wait_deps(grids[it.grid], it, p.progress, i, c, halo, tile, p.wait_limit))
                atomicOr(grids[it.grid].flags, 4u);
        }
        __syncthreads();
        const int ns = c == p.n_chunks - 1 ? p.last_steps : p.K;
        batch_body<N, R, Cell, kFlags | kBodyCg>(grids, items, consts, c & 1, ns, halo, tile,
                                                 step_offset + static_cast<int64_t>(c) * p.K, smem_raw, i);
        __syncthreads();  // every thread's writes of the chunk are done
        if (threadIdx.x == 0) {
            __threadfence();
            st_release(p.progress + i, c + 1);
        }
    }
}

template <int N, typename R, typename Cell>
__global__ void __launch_bounds__(kMaxThreads, 1)
    mln_block_kernel(const __grid_constant__ BlockArgs<R> a, const __grid_constant__ typename Cell::Consts k) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // Launched with a programmatic dependency on the kernel before it in the
    // stream: wait for that grid to complete (its fields and states visible)
    // before any read or write, then let the next launch place its blocks as
    // this grid's blocks exit. Without such a dependency both are no-ops.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    block_body<N, R, Cell>(a, k, static_cast<int64_t>(blockIdx.x), smem_raw);
}

// The adjoint's recomputation: the Strang step with its intermediates traced
// (StrangTraceCell), at most 256 threads a block (the register room the
// trace needs), segment blockIdx.y of a side-by-side launch (0 when
// gridDim.y == 1). Programmatic dependency as in mln_block_kernel.
template <int N, typename R>
__global__ void __launch_bounds__(256, 1)
    mln_trace_kernel(const __grid_constant__ BlockArgs<R> a, const __grid_constant__ StrangConsts<N, R> k) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    {
        const int64_t off = static_cast<int64_t>(blockIdx.y) * a.seg_bytes;
        BlockArgs<R> b = a;
        b.E_in = byte_advance(a.E_in, off);
        b.H_in = byte_advance(a.H_in, off);
        b.s_in = byte_advance(a.s_in, off);
        b.E_out = byte_advance(a.E_out, off);
        b.H_out = byte_advance(a.H_out, off);
        b.s_out = byte_advance(a.s_out, off);
        b.rec_E = byte_advance(a.rec_E, off);
        b.rec_H = byte_advance(a.rec_H, off);
        b.rec_S = byte_advance(a.rec_S, off);
        b.rec_I = byte_advance(a.rec_I, off);
        b.src = a.src ? a.src + static_cast<int64_t>(blockIdx.y) * a.seg_src : nullptr;
        block_body<N, R, StrangTraceCell<N, R>>(b, k, static_cast<int64_t>(blockIdx.x), smem_raw);
    }
}

}  // namespace mln
