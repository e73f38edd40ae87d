// Host FP64 set-up of the adjoint-representation MLN step.
//
// Everything here runs once per context (Secs. 3 and 4 of Riesch &
// Jirauschek): the SU(N) generators, the real matrices M and U and the
// vectors d_eq and v of the adjoint Liouville equation, the field-free
// propagator A0 = exp(M dt/2) with its affine offset, the real eigenbasis T of
// the antisymmetric U with its rotation rates, and the polarisation
// coefficients. The per-cell, per-step work happens on the GPU with these.
#include "setup.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace mln {
namespace {

using CMat = std::vector<cd>;  // N x N, row-major

CMat cmat_from(const double *src, int n) {
    CMat m(static_cast<size_t>(n) * n);
    for (int i = 0; i < n * n; ++i) m[i] = cd(src[2 * i], src[2 * i + 1]);
    return m;
}

CMat cmul(const CMat &a, const CMat &b, int n) {
    CMat c(static_cast<size_t>(n) * n, cd(0, 0));
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            cd aik = a[i * n + k];
            for (int j = 0; j < n; ++j) c[i * n + j] += aik * b[k * n + j];
        }
    return c;
}

CMat cadj(const CMat &a, int n) {
    CMat c(a.size());
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) c[i * n + j] = std::conj(a[j * n + i]);
    return c;
}

cd ctrace(const CMat &a, int n) {
    cd s(0, 0);
    for (int i = 0; i < n; ++i) s += a[i * n + i];
    return s;
}

// Tr{A B} without forming the product.
cd trace_of_product(const CMat &a, const CMat &b, int n) {
    cd s(0, 0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) s += a[i * n + k] * b[k * n + i];
    return s;
}

double max_abs(const CMat &a) {
    double m = 0;
    for (auto &x : a) m = std::max(m, std::abs(x));
    return m;
}

// Apply a superoperator (N^2 x N^2 complex, row-major vec) to X.
CMat superop_apply(const double *G, const CMat &X, int n) {
    const int nn = n * n;
    CMat y(nn, cd(0, 0));
    for (int r = 0; r < nn; ++r) {
        cd s(0, 0);
        for (int c = 0; c < nn; ++c) s += cd(G[2 * (r * nn + c)], G[2 * (r * nn + c) + 1]) * X[c];
        y[r] = s;
    }
    return y;
}

// Generators of SU(N) in the order of Sec. 3: u_jk (j < k, row-major pairs),
// then v_jk, then w_l (l = 1..N-1), with t_jk = |j><k| and
// u_jk = t_jk + t_kj, v_jk = -i (t_jk - t_kj),
// w_l = -sqrt(2/(l(l+1))) (t_11 + ... + t_ll - l t_{l+1,l+1}) (Eq. 7).
std::vector<CMat> make_generators(int n) {
    std::vector<CMat> g;
    std::vector<std::pair<int, int>> pairs;
    for (int j = 0; j < n; ++j)
        for (int k = j + 1; k < n; ++k) pairs.emplace_back(j, k);
    for (auto [j, k] : pairs) {
        CMat u(n * n, cd(0, 0));
        u[j * n + k] = 1.0;
        u[k * n + j] = 1.0;
        g.push_back(u);
    }
    for (auto [j, k] : pairs) {
        CMat v(n * n, cd(0, 0));
        v[j * n + k] = cd(0, -1);
        v[k * n + j] = cd(0, 1);
        g.push_back(v);
    }
    for (int l = 1; l < n; ++l) {
        CMat w(n * n, cd(0, 0));
        double f = -std::sqrt(2.0 / (l * (l + 1.0)));
        for (int m = 0; m < l; ++m) w[m * n + m] = f;
        w[l * n + l] = -f * l;
        g.push_back(w);
    }
    return g;
}

// Eigen-decomposition of a Hermitian matrix by cyclic complex Jacobi
// rotations: A = W diag(ev) W^+. Each rotation first removes the phase of the
// pivot a_pq = r e^{i phi} with diag(1, e^{-i phi}) and then zeroes the real
// pivot with a plane rotation (Rutishauser's stable tangent formula).
void hermitian_eig(const CMat &A_in, int n, std::vector<double> &ev, CMat &W) {
    CMat A = A_in;
    W.assign(static_cast<size_t>(n) * n, cd(0, 0));
    for (int i = 0; i < n; ++i) W[i * n + i] = 1.0;
    double scale = std::max(max_abs(A), 1e-300);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += std::norm(A[p * n + q]);
        if (std::sqrt(off) <= 1e-17 * scale) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                cd apq = A[p * n + q];
                double r = std::abs(apq);
                if (r <= 1e-300) continue;
                cd ph = apq / r;  // e^{i phi}
                double app = A[p * n + p].real(), aqq = A[q * n + q].real();
                double zeta = (aqq - app) / (2.0 * r);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                // J = diag(1, conj(ph)) * [[c, s], [-s, c]] on the (p, q) plane
                CMat J(static_cast<size_t>(n) * n, cd(0, 0));
                for (int i = 0; i < n; ++i) J[i * n + i] = 1.0;
                J[p * n + p] = c;
                J[p * n + q] = s;
                J[q * n + p] = -s * std::conj(ph);
                J[q * n + q] = c * std::conj(ph);
                A = cmul(cadj(J, n), cmul(A, J, n), n);
                W = cmul(W, J, n);
            }
    }
    ev.resize(n);
    for (int i = 0; i < n; ++i) ev[i] = A[i * n + i].real();
    // ascending order
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return ev[a] < ev[b]; });
    std::vector<double> ev2(n);
    CMat W2(W.size());
    for (int c = 0; c < n; ++c) {
        ev2[c] = ev[idx[c]];
        for (int r = 0; r < n; ++r) W2[r * n + c] = W[r * n + idx[c]];
    }
    ev = ev2;
    W = W2;
}

// Real dense helpers (row-major).
using RMat = std::vector<double>;

RMat rmul(const RMat &a, const RMat &b, int n) {
    RMat c(static_cast<size_t>(n) * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            double aik = a[i * n + k];
            for (int j = 0; j < n; ++j) c[i * n + j] += aik * b[k * n + j];
        }
    return c;
}

RMat rtrans(const RMat &a, int n) {
    RMat c(a.size());
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) c[i * n + j] = a[j * n + i];
    return c;
}

std::vector<double> rmatvec(const RMat &a, const std::vector<double> &x, int n) {
    std::vector<double> y(n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) y[i] += a[i * n + j] * x[j];
    return y;
}

double rnorm1(const RMat &a, int n) {
    double best = 0;
    for (int j = 0; j < n; ++j) {
        double s = 0;
        for (int i = 0; i < n; ++i) s += std::fabs(a[i * n + j]);
        best = std::max(best, s);
    }
    return best;
}

// exp(A) of a real n x n matrix: truncated Taylor series with scaling and
// squaring (Moler & Van Loan, "Nineteen dubious ways to compute the
// exponential of a matrix", SIAM Review 45 (2003), methods 1 and 3):
// scale so that ||A/2^s||_1 <= 1/4, sum terms until they stop changing the
// result, square s times.
RMat expm_taylor(const RMat &A, int n) {
    double nrm = rnorm1(A, n);
    int s = 0;
    while (std::ldexp(nrm, -s) > 0.25) ++s;
    RMat B(A.size());
    for (size_t i = 0; i < A.size(); ++i) B[i] = std::ldexp(A[i], -s);
    RMat X(static_cast<size_t>(n) * n, 0.0), term(static_cast<size_t>(n) * n, 0.0);
    for (int i = 0; i < n; ++i) X[i * n + i] = term[i * n + i] = 1.0;
    for (int k = 1; k <= 40; ++k) {
        term = rmul(term, B, n);
        double tn = 0;
        for (auto &t : term) t /= k, tn = std::max(tn, std::fabs(t));
        for (size_t i = 0; i < X.size(); ++i) X[i] += term[i];
        if (tn < 1e-19) break;
    }
    for (int r = 0; r < s; ++r) X = rmul(X, X, n);
    return X;
}

bool finite_all(const double *p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

mln_status adjoint_chain(const mln_params &p, const Setup &s, const double *acc, double *dJ_dmu, double *dJ_dG,
                         std::string &err) {
    const int n = s.N, nn = n * n, D = s.D, q = s.q, Da = D + 1;
    // accumulator layout: Dl (D x D) | b (D) | w (D) | c | T (D x D) | theta (q) | J
    const double *Abar = acc, *bbar = acc + D * D, *wbar = bbar + D, cbar = wbar[D];
    const double *Tbar = wbar + D + 1, *thbar = Tbar + D * D;
    std::vector<CMat> g = make_generators(n);

    // M_bar and d_eq_bar from the augmented propagator [[A0, b], [0, 1]] = exp(X),
    // X = [[M, d_eq], [0, 0]] dt/2. The adjoint of the Frechet derivative of exp
    // at X is the Frechet derivative at X^T, read off the block-triangular
    // exponential exp([[X^T, G], [0, X^T]]) (Van Loan 1978).
    const int D2 = 2 * Da;
    RMat big((size_t)D2 * D2, 0.0);
    const double h = 0.5 * p.dt;
    for (int i = 0; i < D; ++i) {
        for (int j = 0; j < D; ++j) {
            big[j * D2 + i] = s.M[i * D + j] * h;               // X^T, top-left
            big[(Da + j) * D2 + Da + i] = s.M[i * D + j] * h;   // X^T, bottom-right
            big[i * D2 + Da + j] = Abar[i * D + j];             // G = [[A0_bar, b_bar], [0, 0]]
        }
        big[D * D2 + i] = s.d_eq[i] * h;                        // (X^T)_{D, i} = X_{i, D}
        big[(Da + D) * D2 + Da + i] = s.d_eq[i] * h;
        big[i * D2 + Da + D] = bbar[i];
    }
    RMat eb = expm_taylor(big, D2);
    std::vector<double> Mbar((size_t)D * D), deqbar(D);
    for (int i = 0; i < D; ++i) {
        for (int j = 0; j < D; ++j) Mbar[i * D + j] = h * eb[i * D2 + Da + j];
        deqbar[i] = h * eb[i * D2 + Da + D];
    }
    // polarisation coefficients: w_j = N_a/2 sum_k v_k M_kj, c = N_a/2 sum_k v_k d_eq_k
    std::vector<double> vbar(D, 0.0);
    for (int k = 0; k < D; ++k) {
        for (int j = 0; j < D; ++j) {
            Mbar[k * D + j] += 0.5 * p.N_a * s.v[k] * wbar[j];
            vbar[k] += 0.5 * p.N_a * s.M[k * D + j] * wbar[j];
        }
        deqbar[k] += 0.5 * p.N_a * s.v[k] * cbar;
        vbar[k] += 0.5 * p.N_a * s.d_eq[k] * cbar;
    }
    // G: g_jk = Re(1/2 Tr{G(s_k) s_j}), d_eq_j = Re(1/N Tr{G(I) s_j}), and
    // Tr{G(X) Y} = sum_{(a,b), c} G[(a,b), c] vec(X)_c Y_{ba}
    if (dJ_dG) {
        for (int a = 0; a < n; ++a)
            for (int bb = 0; bb < n; ++bb) {
                const int r = a * n + bb;
                for (int cc = 0; cc < nn; ++cc) {
                    cd tot(0, 0);
                    for (int j = 0; j < D; ++j) {
                        const cd sj = g[j][bb * n + a];
                        if (sj == cd(0, 0)) continue;
                        cd inner(0, 0);
                        for (int k = 0; k < D; ++k) inner += Mbar[j * D + k] * 0.5 * g[k][cc];
                        const int ci = cc / n, cj = cc % n;
                        if (ci == cj) inner += deqbar[j] / n;
                        tot += inner * sj;
                    }
                    const cd gam = std::conj(tot);
                    dJ_dG[2 * (r * nn + cc)] = gam.real();
                    dJ_dG[2 * (r * nn + cc) + 1] = gam.imag();
                }
            }
    }
    if (!dJ_dmu) return MLN_OK;
    // mu: v_k = Tr{mu s_k}; T and theta from mu = W diag(m) W^+ by first-order
    // perturbation: dm_a = Delta_aa, dW = W C, C_ca = Delta_ca / (m_a - m_c)
    // (c != a), C_aa = 0, Delta = W^+ dmu W. (A phase change of an eigenvector
    // turns T within its planes, which commutes with the plane rotations, so the
    // choice C_aa = 0 does not change the result.)
    double mscale = 1e-300;
    for (double m : s.mev) mscale = std::max(mscale, std::fabs(m));
    for (int a = 0; a < n; ++a)
        for (int c = a + 1; c < n; ++c)
            if (std::fabs(s.mev[a] - s.mev[c]) < 1e-9 * mscale) {
                err = "dipole operator has (nearly) degenerate eigenvalues: its gradient is not defined this way";
                return MLN_ENUMERIC;
            }
    const CMat &W = s.Wmu;
    const CMat Wh = cadj(W, n);
    std::vector<CMat> dirs;
    for (int l = 0; l < n; ++l) {
        CMat e(nn, cd(0, 0));
        e[l * n + l] = 1.0;
        dirs.push_back(e);
    }
    for (int j = 0; j < n; ++j)
        for (int k = j + 1; k < n; ++k) {
            CMat e(nn, cd(0, 0));
            e[j * n + k] = 1.0;
            e[k * n + j] = 1.0;
            dirs.push_back(e);
        }
    for (int j = 0; j < n; ++j)
        for (int k = j + 1; k < n; ++k) {
            CMat e(nn, cd(0, 0));
            e[j * n + k] = cd(0, 1);
            e[k * n + j] = cd(0, -1);
            dirs.push_back(e);
        }
    auto coords = [&](const CMat &X, int j) { return 0.5 * trace_of_product(X, g[j], n).real(); };
    for (size_t di = 0; di < dirs.size(); ++di) {
        const CMat &dmu = dirs[di];
        CMat Delta = cmul(Wh, cmul(dmu, W, n), n);
        CMat C(nn, cd(0, 0));
        std::vector<double> dm(n);
        for (int a = 0; a < n; ++a) {
            dm[a] = Delta[a * n + a].real();
            for (int c = 0; c < n; ++c)
                if (c != a) C[c * n + a] = Delta[c * n + a] / (s.mev[a] - s.mev[c]);
        }
        CMat Ch = cadj(C, n);
        double dJ = 0;
        // T columns of the planes (only their gradient is non-zero)
        int k = 0;
        for (int a = 0; a < n; ++a)
            for (int b = a + 1; b < n; ++b, ++k) {
                CMat X(nn, cd(0, 0)), Y(nn, cd(0, 0));
                X[a * n + b] = 1.0;
                X[b * n + a] = 1.0;
                Y[a * n + b] = cd(0, -1);
                Y[b * n + a] = cd(0, 1);
                for (int col = 0; col < 2; ++col) {
                    const CMat &E0 = col == 0 ? X : Y;
                    CMat inner = cmul(C, E0, n), tmp = cmul(E0, Ch, n);
                    for (int t = 0; t < nn; ++t) inner[t] += tmp[t];
                    CMat dX = cmul(W, cmul(inner, Wh, n), n);
                    for (int j = 0; j < D; ++j) dJ += Tbar[j * D + 2 * k + col] * coords(dX, j);
                }
                dJ += thbar[k] * (dm[a] - dm[b]) / kHbar;
            }
        for (int j = 0; j < D; ++j) dJ += vbar[j] * trace_of_product(dmu, g[j], n).real();
        dJ_dmu[di] = dJ;
    }
    return MLN_OK;
}

int64_t state_stride(const mln_params &p) {
    int64_t nm = p.medium_end - p.medium_begin;
    return (nm + 63) / 64 * 64;
}

mln_status validate(const mln_params &p, std::string &err) {
    if (p.N < 2 || p.N > 8) {
        err = "N must be in [2, 8]";
        return MLN_EINVAL;
    }
    if (p.N > MLN_MAX_N) {
        err = "N = " + std::to_string(p.N) + " is above the compiled maximum " +
              std::to_string(MLN_MAX_N);
        return MLN_EUNSUPPORTED;
    }
    if (!p.H0 || !p.mu || !p.rho0) {
        err = "H0, mu and rho0 are required";
        return MLN_EINVAL;
    }
    if (p.precision != MLN_FP64 && p.precision != MLN_FP32) {
        err = "precision must be MLN_FP64 or MLN_FP32";
        return MLN_EINVAL;
    }
    if (p.form != MLN_FORM_STRANG && p.form != MLN_FORM_MERGED && p.form != MLN_FORM_RODRIGUES &&
        p.form != MLN_FORM_ROTATED) {
        err = "form must be MLN_FORM_STRANG, MLN_FORM_MERGED, MLN_FORM_RODRIGUES or MLN_FORM_ROTATED";
        return MLN_EINVAL;
    }
    if (p.form == MLN_FORM_ROTATED &&
        ((p.kernel != MLN_KERNEL_AUTO && p.kernel != MLN_KERNEL_JIT && p.kernel != MLN_KERNEL_TENSOR &&
          p.kernel != MLN_KERNEL_DF32) ||
         p.maxwell != MLN_MAXWELL_FDTD)) {
        err = "MLN_FORM_ROTATED runs on the run-time compiled, double-float or tensor-core kernel (MLN_KERNEL_AUTO, "
              "MLN_KERNEL_JIT, MLN_KERNEL_DF32 or MLN_KERNEL_TENSOR) with MLN_MAXWELL_FDTD";
        return MLN_EINVAL;
    }
    if (p.form == MLN_FORM_RODRIGUES && p.N > 4) {
        err = "MLN_FORM_RODRIGUES is built for N <= 4";
        return MLN_EUNSUPPORTED;
    }
    if (p.boundary != MLN_BC_PERIODIC && p.boundary != MLN_BC_OPEN) {
        err = "boundary must be MLN_BC_PERIODIC or MLN_BC_OPEN";
        return MLN_EINVAL;
    }
    if (p.source_kind < MLN_SRC_NONE || p.source_kind > MLN_SRC_SOFT) {
        err = "source_kind must be MLN_SRC_NONE, MLN_SRC_HARD or MLN_SRC_SOFT";
        return MLN_EINVAL;
    }
    if (p.n_cells < 4) {
        err = "n_cells must be >= 4";
        return MLN_EINVAL;
    }
    if (p.medium_begin < 0 || p.medium_end < p.medium_begin || p.medium_end > p.n_cells) {
        err = "need 0 <= medium_begin <= medium_end <= n_cells";
        return MLN_EINVAL;
    }
    if (p.boundary == MLN_BC_OPEN && p.medium_end > p.n_cells - 1) {
        err = "with MLN_BC_OPEN the last cell (Mur boundary) must be vacuum";
        return MLN_EINVAL;
    }
    if (p.source_kind != MLN_SRC_NONE && (p.source_cell < 0 || p.source_cell >= p.n_cells)) {
        err = "source_cell out of range";
        return MLN_EINVAL;
    }
    const double sc[] = {p.N_a, p.dx, p.dt, p.eps_r, p.mu_r, p.sigma};
    if (!finite_all(sc, 6) || p.dx <= 0 || p.dt <= 0 || p.eps_r <= 0 || p.mu_r <= 0 ||
        p.sigma < 0 || p.N_a < 0) {
        err = "need finite dx, dt, eps_r, mu_r > 0 and sigma, N_a >= 0";
        return MLN_EINVAL;
    }
    double cv = 1.0 / std::sqrt(kEps0 * p.eps_r * kMu0 * p.mu_r);
    if (cv * p.dt / p.dx > 1.0 + 1e-12) {
        err = "Courant number c dt / dx exceeds 1";
        return MLN_EINVAL;
    }
    if (p.block_steps < 0 || p.block_steps > 64) {
        err = "block_steps must be in [0, 64]";
        return MLN_EINVAL;
    }
    if (p.maxwell != MLN_MAXWELL_FDTD && p.maxwell != MLN_MAXWELL_PSTD) {
        err = "maxwell must be MLN_MAXWELL_FDTD or MLN_MAXWELL_PSTD";
        return MLN_EINVAL;
    }
    if (p.maxwell == MLN_MAXWELL_PSTD) {
        const bool pow2 = p.n_cells >= 16 && p.n_cells <= (int64_t(1) << 24) && (p.n_cells & (p.n_cells - 1)) == 0;
        if (p.boundary != MLN_BC_PERIODIC || !pow2) {
            err = "MLN_MAXWELL_PSTD needs a periodic grid of 2^k cells, 16 <= n_cells <= 2^24";
            return MLN_EINVAL;
        }
        if (p.kernel != MLN_KERNEL_AUTO && p.kernel != MLN_KERNEL_REGISTER && p.kernel != MLN_KERNEL_SPARSE) {
            err = "MLN_MAXWELL_PSTD runs with kernel MLN_KERNEL_AUTO, MLN_KERNEL_REGISTER or MLN_KERNEL_SPARSE";
            return MLN_EINVAL;
        }
    }
    if (p.kernel < MLN_KERNEL_AUTO || p.kernel > MLN_KERNEL_DF32) {
        err = "kernel must be MLN_KERNEL_AUTO, MLN_KERNEL_REGISTER, MLN_KERNEL_SPARSE, MLN_KERNEL_JIT, "
              "MLN_KERNEL_TENSOR or MLN_KERNEL_DF32";
        return MLN_EINVAL;
    }
    if (p.kernel == MLN_KERNEL_DF32 && (p.precision != MLN_FP64 ||
                                        (p.form != MLN_FORM_MERGED && p.form != MLN_FORM_ROTATED) ||
                                        p.maxwell != MLN_MAXWELL_FDTD)) {
        err = "MLN_KERNEL_DF32 needs MLN_FP64, MLN_FORM_MERGED or MLN_FORM_ROTATED, and MLN_MAXWELL_FDTD";
        return MLN_EINVAL;
    }
    if (p.kernel == MLN_KERNEL_TENSOR &&
        (p.precision != MLN_FP32 || (p.form != MLN_FORM_MERGED && p.form != MLN_FORM_ROTATED) || p.N < 5)) {
        err = "MLN_KERNEL_TENSOR needs MLN_FP32, MLN_FORM_MERGED or MLN_FORM_ROTATED, and N = 5 or 6";
        return MLN_EINVAL;
    }
    if (p.kernel == MLN_KERNEL_TENSOR && p.block_steps > 32) {
        err = "MLN_KERNEL_TENSOR fuses at most 32 steps per launch";
        return MLN_EINVAL;
    }
    if (p.kernel == MLN_KERNEL_JIT && p.form != MLN_FORM_MERGED && p.form != MLN_FORM_ROTATED) {
        err = "MLN_KERNEL_JIT needs MLN_FORM_MERGED or MLN_FORM_ROTATED";
        return MLN_EINVAL;
    }
    if (p.kernel == MLN_KERNEL_SPARSE && (p.precision != MLN_FP64 || p.form != MLN_FORM_MERGED)) {
        err = "MLN_KERNEL_SPARSE needs MLN_FP64 and MLN_FORM_MERGED";
        return MLN_EINVAL;
    }
    if (p.tile_cells < 0) {
        err = "tile_cells must be >= 0";
        return MLN_EINVAL;
    }
    const int n = p.N, nn = n * n;
    if (!finite_all(p.H0, 2 * nn) || !finite_all(p.mu, 2 * nn) || !finite_all(p.rho0, 2 * nn) ||
        (p.G && !finite_all(p.G, 2 * (size_t)nn * nn))) {
        err = "non-finite entries in H0, mu, rho0 or G";
        return MLN_EINVAL;
    }
    auto herm_err = [&](const CMat &a) {
        double m = 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) m = std::max(m, std::abs(a[i * n + j] - std::conj(a[j * n + i])));
        return m;
    };
    CMat H0 = cmat_from(p.H0, n), mu = cmat_from(p.mu, n), rho0 = cmat_from(p.rho0, n);
    if (herm_err(H0) > 1e-12 * max_abs(H0) || herm_err(mu) > 1e-12 * max_abs(mu)) {
        err = "H0 and mu must be Hermitian";
        return MLN_EINVAL;
    }
    if (herm_err(rho0) > 1e-12 || std::abs(ctrace(rho0, n) - 1.0) > 1e-12) {
        err = "rho0 must be Hermitian with unit trace";
        return MLN_EINVAL;
    }
    std::vector<double> ev;
    CMat W;
    hermitian_eig(rho0, n, ev, W);
    if (ev[0] < -1e-12) {
        err = "rho0 must be positive semidefinite";
        return MLN_EINVAL;
    }
    if (p.G) {
        double gmax = 0;
        for (size_t i = 0; i < 2 * (size_t)nn * nn; ++i) gmax = std::max(gmax, std::fabs(p.G[i]));
        double tol = 1e-12 * std::max(gmax, 1e-300);
        // trace preservation: sum_l G[(l,l), c] = 0 for every column c
        for (int c = 0; c < nn; ++c) {
            cd s(0, 0);
            for (int l = 0; l < n; ++l) {
                int r = l * n + l;
                s += cd(p.G[2 * (r * nn + c)], p.G[2 * (r * nn + c) + 1]);
            }
            if (std::abs(s) > tol * n) {
                err = "G must preserve the trace";
                return MLN_EINVAL;
            }
        }
        // Hermiticity preservation: G[(j,k),(l,m)] = conj(G[(k,j),(m,l)])
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k)
                for (int l = 0; l < n; ++l)
                    for (int m = 0; m < n; ++m) {
                        int r1 = j * n + k, c1 = l * n + m, r2 = k * n + j, c2 = m * n + l;
                        cd a(p.G[2 * (r1 * nn + c1)], p.G[2 * (r1 * nn + c1) + 1]);
                        cd b(p.G[2 * (r2 * nn + c2)], p.G[2 * (r2 * nn + c2) + 1]);
                        if (std::abs(a - std::conj(b)) > tol) {
                            err = "G must map Hermitian matrices to Hermitian matrices";
                            return MLN_EINVAL;
                        }
                    }
    }
    return MLN_OK;
}

mln_status build_setup(const mln_params &p, Setup &s, std::string &err) {
    const int n = p.N, nn = n * n, D = nn - 1, q = n * (n - 1) / 2;
    s.N = n;
    s.D = D;
    s.q = q;
    std::vector<CMat> g = make_generators(n);
    s.gen.clear();
    for (auto &m : g) s.gen.insert(s.gen.end(), m.begin(), m.end());

    CMat H0 = cmat_from(p.H0, n), mu = cmat_from(p.mu, n), rho0 = cmat_from(p.rho0, n);
    auto comm = [&](const CMat &a, const CMat &b) {
        CMat ab = cmul(a, b, n), ba = cmul(b, a, n);
        for (size_t i = 0; i < ab.size(); ++i) ab[i] -= ba[i];
        return ab;
    };
    auto G_of = [&](const CMat &X) {
        if (!p.G) return CMat(nn, cd(0, 0));
        return superop_apply(p.G, X, n);
    };

    // d_j = Tr{rho s_j} (Eq. 6), v_k = Tr{mu s_k} (Eq. 15)
    s.d0.assign(D, 0.0);
    s.v.assign(D, 0.0);
    for (int j = 0; j < D; ++j) {
        s.d0[j] = trace_of_product(rho0, g[j], n).real();
        s.v[j] = trace_of_product(mu, g[j], n).real();
    }
    // m_jk = (i/2hbar) Tr{H0 [s_j, s_k]} + g_jk,  g_jk = 1/2 Tr{G(s_k) s_j},
    // u_jk = -(i/2hbar) Tr{mu [s_j, s_k]}   (Eqs. 11 and 13)
    s.M.assign((size_t)D * D, 0.0);
    s.U.assign((size_t)D * D, 0.0);
    double imag_max = 0, real_max = 1e-300;
    std::vector<CMat> Gs(D);
    for (int k = 0; k < D; ++k) Gs[k] = G_of(g[k]);
    for (int j = 0; j < D; ++j)
        for (int k = 0; k < D; ++k) {
            CMat cjk = comm(g[j], g[k]);
            cd m = cd(0, 0.5 / kHbar) * trace_of_product(H0, cjk, n) + 0.5 * trace_of_product(Gs[k], g[j], n);
            cd u = cd(0, -0.5 / kHbar) * trace_of_product(mu, cjk, n);
            s.M[j * D + k] = m.real();
            s.U[j * D + k] = u.real();
            imag_max = std::max({imag_max, std::fabs(m.imag()), std::fabs(u.imag())});
            real_max = std::max({real_max, std::fabs(m.real()), std::fabs(u.real())});
        }
    if (imag_max > 1e-10 * real_max) {
        err = "M or U came out complex: check the inputs";
        return MLN_ENUMERIC;
    }
    // d_eq_j = N^-1 Tr{G(I) s_j} (Eq. 12)
    s.d_eq.assign(D, 0.0);
    {
        CMat I(nn, cd(0, 0));
        for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
        CMat GI = G_of(I);
        for (int j = 0; j < D; ++j) s.d_eq[j] = trace_of_product(GI, g[j], n).real() / n;
    }

    // A0 and b from the augmented flow exp([[M, d_eq], [0, 0]] dt/2): the
    // affine solution of Eq. 19 over dt/2, defined whether or not M is
    // invertible (equal to A0 (d + d_in) - d_in when it is).
    const int Da = D + 1;
    RMat Ma((size_t)Da * Da, 0.0);
    for (int i = 0; i < D; ++i) {
        for (int j = 0; j < D; ++j) Ma[i * Da + j] = s.M[i * D + j] * 0.5 * p.dt;
        Ma[i * Da + D] = s.d_eq[i] * 0.5 * p.dt;
    }
    RMat Ea = expm_taylor(Ma, Da);
    RMat Man(Ma.size());
    for (size_t i = 0; i < Ma.size(); ++i) Man[i] = -Ma[i];
    RMat Eai = expm_taylor(Man, Da);
    s.A0.assign((size_t)D * D, 0.0);
    s.A0inv.assign((size_t)D * D, 0.0);
    s.b.assign(D, 0.0);
    s.binv.assign(D, 0.0);
    for (int i = 0; i < D; ++i) {
        for (int j = 0; j < D; ++j) {
            s.A0[i * D + j] = Ea[i * Da + j];
            s.A0inv[i * D + j] = Eai[i * Da + j];
        }
        s.b[i] = Ea[i * Da + D];
        s.binv[i] = Eai[i * Da + D];
    }

    // Real eigenbasis of U (Sec. 4.2, Eq. 26). U d is the coordinate vector of
    // (i/hbar)[mu, X] for X = 1/2 sum d_j s_j, so U is diagonalised by the
    // eigen-decomposition mu = W diag(m) W^+: for a < b the pair
    // X_ab = W(|a><b| + |b><a|)W^+, Y_ab = W(-i)(|a><b| - |b><a|)W^+ spans an
    // invariant plane of U with eigenvalues +-i (m_a - m_b)/hbar, and the
    // images W w_l W^+ of the diagonal generators span its null space. The
    // coordinates x_j = Tr{X s_j}/2 of these matrices are orthonormal.
    std::vector<double> mev;
    CMat Wm;
    hermitian_eig(mu, n, mev, Wm);
    s.Wmu = Wm;
    s.mev = mev;
    CMat Wh = cadj(Wm, n);
    s.T.assign((size_t)D * D, 0.0);
    s.theta.assign(q, 0.0);
    s.psi.assign(n - 1, 0.0);
    for (int a = 0; a < n - 1; ++a) s.psi[a] = (mev[a] - mev[n - 1]) / kHbar;
    auto put_col = [&](int col, const CMat &X) {
        for (int j = 0; j < D; ++j) s.T[j * D + col] = 0.5 * trace_of_product(X, g[j], n).real();
    };
    int pidx = 0;
    for (int a = 0; a < n; ++a)
        for (int b = a + 1; b < n; ++b) {
            CMat X(nn, cd(0, 0)), Y(nn, cd(0, 0));
            X[a * n + b] = 1.0;
            X[b * n + a] = 1.0;
            Y[a * n + b] = cd(0, -1);
            Y[b * n + a] = cd(0, 1);
            put_col(2 * pidx, cmul(Wm, cmul(X, Wh, n), n));
            put_col(2 * pidx + 1, cmul(Wm, cmul(Y, Wh, n), n));
            s.theta[pidx] = (mev[a] - mev[b]) / kHbar;
            ++pidx;
        }
    for (int l = 0; l < n - 1; ++l) put_col(2 * q + l, cmul(Wm, cmul(g[2 * q + l], Wh, n), n));

    // Check: T^T T = I and T^T U T = block-diag [[0, theta], [-theta, 0]].
    RMat Tt = rtrans(s.T, D);
    RMat TtT = rmul(Tt, s.T, D);
    RMat B = rmul(Tt, rmul(s.U, s.T, D), D);
    double orth = 0, resid = 0, unorm = 1e-300;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            orth = std::max(orth, std::fabs(TtT[i * D + j] - (i == j ? 1.0 : 0.0)));
            unorm = std::max(unorm, std::fabs(s.U[i * D + j]));
            double want = 0;
            if (i < 2 * q && j < 2 * q && i / 2 == j / 2 && i != j) want = (i % 2 == 0) ? s.theta[i / 2] : -s.theta[i / 2];
            resid = std::max(resid, std::fabs(B[i * D + j] - want));
        }
    s.resid_orth = orth;
    s.resid_eig = resid / unorm;
    if (orth > 1e-12 || resid > 1e-12 * unorm) {
        err = "eigen-decomposition of U failed its residual check";
        return MLN_ENUMERIC;
    }

    // dP/dt = N_a/2 v^T (M d + d_eq) = w . d + c (Eq. 17)
    s.w.assign(D, 0.0);
    for (int j = 0; j < D; ++j) {
        double acc = 0;
        for (int k = 0; k < D; ++k) acc += s.v[k] * s.M[k * D + j];
        s.w[j] = 0.5 * p.N_a * acc;
    }
    {
        double acc = 0;
        for (int k = 0; k < D; ++k) acc += s.v[k] * s.d_eq[k];
        s.c = 0.5 * p.N_a * acc;
    }

    // Merged form (state y = d' = A0 d + b after the first half-step of Eq. 23a):
    // y'' = exp(U E dt) y; dP/dt = w . (A0 y'' + b) + c = (A0^T w) . y'' + (w . b + c);
    // the next state is A0 (A0 y'' + b) + b = y'' + (A0^2 - I) y'' + (A0 b + b).
    RMat A0sq = rmul(s.A0, s.A0, D);
    s.C1 = A0sq;
    for (int i = 0; i < D; ++i) s.C1[i * D + i] -= 1.0;
    s.b2 = rmatvec(s.A0, s.b, D);
    for (int i = 0; i < D; ++i) s.b2[i] += s.b[i];
    s.wm = rmatvec(rtrans(s.A0, D), s.w, D);
    s.cm = s.c;
    for (int i = 0; i < D; ++i) s.cm += s.w[i] * s.b[i];

    // Rotated form (state z = T^T y, T orthogonal): z'' = R(E) z on the plane
    // pairs; dP/dt = (T^T wm) . z'' + cm; the next state is
    // T^T (y'' + C1 y'' + b2) = z'' + (T^T C1 T) z'' + T^T b2.
    s.C1z = rmul(Tt, rmul(s.C1, s.T, D), D);
    s.cz = rmatvec(Tt, s.b2, D);
    s.wz = rmatvec(Tt, s.wm, D);

    // State <-> adjoint vector maps.
    s.Sd.assign((size_t)D * D, 0.0);
    s.sd0.assign(D, 0.0);
    s.Sp.assign((size_t)D * D, 0.0);
    s.sp0.assign(D, 0.0);
    if (p.form == MLN_FORM_MERGED) {
        // d = A0^-1 (y - b) = A0inv y + binv;  y = A0 d + b
        s.Sd = s.A0inv;
        s.sd0 = s.binv;
        s.Sp = s.A0;
        s.sp0 = s.b;
    } else if (p.form == MLN_FORM_ROTATED) {
        // d = A0inv T z + binv;  z = T^T A0 d + T^T b
        s.Sd = rmul(s.A0inv, s.T, D);
        s.sd0 = s.binv;
        s.Sp = rmul(Tt, s.A0, D);
        s.sp0 = rmatvec(Tt, s.b, D);
    } else {
        for (int i = 0; i < D; ++i) s.Sd[i * D + i] = s.Sp[i * D + i] = 1.0;
    }

    // rho = I/N + 1/2 sum_j d_j s_j (Eq. 6) as rho_c + Z d over interleaved re/im.
    s.rho_c.assign(2 * nn, 0.0);
    s.Z.assign((size_t)2 * nn * D, 0.0);
    for (int i = 0; i < n; ++i) s.rho_c[2 * (i * n + i)] = 1.0 / n;
    for (int e = 0; e < nn; ++e)
        for (int j = 0; j < D; ++j) {
            s.Z[(2 * e) * D + j] = 0.5 * g[j][e].real();
            s.Z[(2 * e + 1) * D + j] = 0.5 * g[j][e].imag();
        }
    return MLN_OK;
}

}  // namespace mln
