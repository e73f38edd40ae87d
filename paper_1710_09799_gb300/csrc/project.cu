// Positivity projection of the medium state (optional, FP64, off the step
// path). In the adjoint representation trace and Hermiticity of rho hold by
// construction (Eq. 6: real coefficients of traceless Hermitian generators),
// so the only property that rounding can break is rho >= 0. For every cell
// whose rho has a negative eigenvalue, rho is replaced by the nearest unit-
// trace positive semidefinite matrix in the Frobenius norm: the eigenvalues
// are projected onto the probability simplex (sort, then subtract the one
// threshold that leaves the positive part summing to one), the eigenvectors
// kept. The Hermitian eigen-decomposition is cyclic Jacobi with complex
// rotations. Cells whose smallest eigenvalue is at least -16 N u (u the unit
// roundoff of the state's precision: a zero eigenvalue after rounding) are
// left bit for bit as they were.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "ctx.h"
#include "mln.h"
#include "setup.h"

namespace {

constexpr int kMaxN = MLN_MAX_N;

struct Cx {
    double re, im;
};

__device__ __forceinline__ Cx cmul(Cx a, Cx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ Cx cconj(Cx a) { return {a.re, -a.im}; }

// a (n x n Hermitian, row-major) -> eigenvalues on its diagonal, v the
// eigenvectors as columns.
__device__ void jacobi_hermitian(int n, Cx (&a)[kMaxN][kMaxN], Cx (&v)[kMaxN][kMaxN]) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) v[i][j] = {i == j ? 1.0 : 0.0, 0.0};
    double scale = 0.0;
    for (int i = 0; i < n; ++i) scale += a[i][i].re * a[i][i].re;
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += a[p][q].re * a[p][q].re + a[p][q].im * a[p][q].im;
        if (off <= 1e-32 * (scale + 1e-300)) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double m = hypot(a[p][q].re, a[p][q].im);
                if (m == 0.0) continue;
                // a_pq = m e^{i phi}; U = diag(1, e^{-i phi}) R with the real rotation R
                // that annihilates the off-diagonal of [[a_pp, m], [m, a_qq]]
                const Cx ph = {a[p][q].re / m, a[p][q].im / m};  // e^{i phi}
                const double tau = (a[q][q].re - a[p][p].re) / (2.0 * m);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                const Cx ec = cconj(ph);  // e^{-i phi}
                // columns: (A U)_kp = c A_kp - s e^{-i phi} A_kq; (A U)_kq = s A_kp + c e^{-i phi} A_kq
                for (int k = 0; k < n; ++k) {
                    const Cx akp = a[k][p], akq = cmul(ec, a[k][q]);
                    a[k][p] = {c * akp.re - s * akq.re, c * akp.im - s * akq.im};
                    a[k][q] = {s * akp.re + c * akq.re, s * akp.im + c * akq.im};
                    const Cx vkp = v[k][p], vkq = cmul(ec, v[k][q]);
                    v[k][p] = {c * vkp.re - s * vkq.re, c * vkp.im - s * vkq.im};
                    v[k][q] = {s * vkp.re + c * vkq.re, s * vkp.im + c * vkq.im};
                }
                // rows: (U^+ M)_pk = c M_pk - s e^{i phi} M_qk; (U^+ M)_qk = s M_pk + c e^{i phi} M_qk
                for (int k = 0; k < n; ++k) {
                    const Cx mpk = a[p][k], mqk = cmul(ph, a[q][k]);
                    a[p][k] = {c * mpk.re - s * mqk.re, c * mpk.im - s * mqk.im};
                    a[q][k] = {s * mpk.re + c * mqk.re, s * mpk.im + c * mqk.im};
                }
                a[p][q] = a[q][p] = {0.0, 0.0};
                a[p][p].im = a[q][q].im = 0.0;
            }
    }
}

// Euclidean projection of lam[0..n) onto {x >= 0, sum x = 1}.
__device__ void simplex_project(int n, double (&lam)[kMaxN]) {
    double u[kMaxN];
    for (int i = 0; i < n; ++i) u[i] = lam[i];
    for (int i = 1; i < n; ++i)  // descending insertion sort
        for (int j = i; j > 0 && u[j] > u[j - 1]; --j) {
            const double t = u[j];
            u[j] = u[j - 1];
            u[j - 1] = t;
        }
    double sum = 0.0, theta = 0.0;
    for (int k = 0; k < n; ++k) {
        sum += u[k];
        const double th = (sum - 1.0) / (k + 1);
        if (u[k] - th > 0.0) theta = th;
    }
    for (int i = 0; i < n; ++i) lam[i] = fmax(lam[i] - theta, 0.0);
}

// rho rows (2 N^2: re, im of rho_ab, row-major) = tab_rho[rows x D] state + offsets,
// d_j = Re Tr(rho s_j) = sum_ab Re(rho_ab (s_j)_ba) from gen (D x N x N complex),
// state = tab_in[D x D] d + offsets.
template <typename R>
__global__ void project_kernel(R *__restrict__ state, int64_t stride, int64_t count, int N, int D,
                               const double *__restrict__ tab_rho, const double *__restrict__ gen,
                               const double *__restrict__ tab_in, double tol,
                               unsigned long long *__restrict__ changed) {
    const int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (c >= count) return;
    const int rows = 2 * N * N;
    double x[kMaxN * kMaxN - 1];
    for (int k = 0; k < D; ++k) x[k] = static_cast<double>(state[k * stride + c]);
    Cx a[kMaxN][kMaxN], v[kMaxN][kMaxN];
    for (int r = 0; r < N * N; ++r) {
        double re = tab_rho[rows * D + 2 * r], im = tab_rho[rows * D + 2 * r + 1];
        for (int k = 0; k < D; ++k) {
            re += tab_rho[(2 * r) * D + k] * x[k];
            im += tab_rho[(2 * r + 1) * D + k] * x[k];
        }
        a[r / N][r % N] = {re, im};
    }
    // Hermitian part (exact up to rounding already)
    for (int i = 0; i < N; ++i)
        for (int j = i; j < N; ++j) {
            const Cx h = {0.5 * (a[i][j].re + a[j][i].re), 0.5 * (a[i][j].im - a[j][i].im)};
            a[i][j] = h;
            a[j][i] = cconj(h);
        }
    Cx w[kMaxN][kMaxN];
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) w[i][j] = a[i][j];
    jacobi_hermitian(N, w, v);
    double lam[kMaxN];
    double lmin = 1e300;
    for (int i = 0; i < N; ++i) {
        lam[i] = w[i][i].re;
        lmin = fmin(lmin, lam[i]);
    }
    if (!(lmin < -tol)) return;  // rho >= 0 up to rounding: untouched
    simplex_project(N, lam);
    // rho' = V diag(lam) V^+
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            Cx s = {0.0, 0.0};
            for (int k = 0; k < N; ++k) {
                const Cx t = cmul(v[i][k], cconj(v[j][k]));
                s.re += lam[k] * t.re;
                s.im += lam[k] * t.im;
            }
            a[i][j] = s;
        }
    double d[kMaxN * kMaxN - 1];
    for (int j = 0; j < D; ++j) {
        double acc = 0.0;
        const double *g = gen + static_cast<size_t>(j) * 2 * N * N;
        for (int p = 0; p < N; ++p)
            for (int q = 0; q < N; ++q) {
                const Cx sqp = {g[2 * (q * N + p)], g[2 * (q * N + p) + 1]};
                acc += a[p][q].re * sqp.re - a[p][q].im * sqp.im;
            }
        d[j] = acc;
    }
    for (int k = 0; k < D; ++k) {
        double acc = tab_in[D * D + k];
        for (int j = 0; j < D; ++j) acc += tab_in[k * D + j] * d[j];
        state[k * stride + c] = static_cast<R>(acc);
    }
    atomicAdd(changed, 1ull);
}

}  // namespace

extern "C" mln_status mln_project_positive(mln_ctx *c, int64_t *n_projected) {
    if (!c) return MLN_EINVAL;
    if (n_projected) *n_projected = 0;
    if (c->n_med == 0) return MLN_OK;
    const int N = c->p.N, D = c->D;
    // generators (D x N x N complex) in the ordering of the set-up
    const size_t gbytes = static_cast<size_t>(D) * 2 * N * N * sizeof(double);
    double *gen = nullptr;
    unsigned long long *dcount = nullptr, hcount = 0;
    mln_status st = MLN_OK;
    std::vector<double> g(static_cast<size_t>(D) * 2 * N * N);
    for (size_t i = 0; i < c->s.gen.size() && i < g.size() / 2; ++i) {
        g[2 * i] = c->s.gen[i].real();
        g[2 * i + 1] = c->s.gen[i].imag();
    }
    cudaError_t e = cudaMalloc(&gen, gbytes);
    if (e == cudaSuccess) e = cudaMalloc(&dcount, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpyAsync(gen, g.data(), gbytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) {
        const unsigned blocks = static_cast<unsigned>((c->n_med + 127) / 128);
        // eigenvalues above -16 N u (u: unit roundoff of the state) are rounding of a zero
        const double u = c->p.precision == MLN_FP64 ? 0x1p-53 : 0x1p-24;
        const double tol = 16.0 * N * u;
        if (c->p.precision == MLN_FP64)
            project_kernel<double><<<blocks, 128, 0, c->stream>>>(static_cast<double *>(c->st[0]), c->stride, c->n_med,
                                                                  N, D, c->tab_rho, gen, c->tab_in, tol, dcount);
        else
            project_kernel<float><<<blocks, 128, 0, c->stream>>>(static_cast<float *>(c->st[0]), c->stride, c->n_med,
                                                                 N, D, c->tab_rho, gen, c->tab_in, tol, dcount);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hcount, dcount, sizeof(hcount), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("mln_project_positive: ") + cudaGetErrorString(e);
        st = MLN_ECUDA;
    } else if (n_projected) {
        *n_projected = static_cast<int64_t>(hcount);
    }
    cudaFree(gen);
    cudaFree(dcount);
    return st;
}
