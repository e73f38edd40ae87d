// Host FP64 set-up of the adjoint-representation MLN step (internal header).
#pragma once

#include <complex>
#include <string>
#include <vector>

#include "mln.h"

namespace mln {

using cd = std::complex<double>;

constexpr double kHbar = 1.054571817e-34;   // J s (CODATA 2018)
constexpr double kEps0 = 8.8541878128e-12;  // F/m
constexpr double kMu0 = 1.25663706212e-6;   // H/m

struct Setup {
    int N = 0, D = 0, q = 0;
    std::vector<cd> gen;                  // D generators, N x N each (Sec. 3)
    std::vector<double> M, U;             // D x D (Eq. 13)
    std::vector<double> d_eq, v;          // D (Eqs. 12, 15)
    std::vector<double> A0, b;            // exp(M dt/2) and its affine offset (Eq. 23)
    std::vector<double> A0inv, binv;      // exp(-M dt/2) of the same affine flow
    std::vector<double> T, theta;         // real eigenbasis of U (Eq. 26), plane rotation rates
    std::vector<double> psi;              // (m_a - m_{N-1})/hbar, a < N-1: base rates of the planes
    std::vector<cd> Wmu;                  // eigenvectors of mu (columns), N x N
    std::vector<double> mev;              // eigenvalues of mu, ascending
    std::vector<double> w;                // N_a/2 M^T v  (Eq. 17)
    double c = 0;                         // N_a/2 v^T d_eq
    std::vector<double> d0;               // adjoint vector of rho0 (Eq. 6)
    // merged form: state y = A0 d + b; C1 = A0^2 - I, b2 = A0 b + b, wm = A0^T w, cm = w . b + c
    std::vector<double> C1, b2, wm;
    double cm = 0;
    // rotated form: state z = T^T y; C1z = T^T C1 T, cz = T^T b2, wz = T^T wm
    std::vector<double> C1z, cz, wz;
    // device state -> adjoint vector d = sd0 + Sd state, and back state = sp0 + Sp d
    std::vector<double> Sd, sd0, Sp, sp0;
    // rho (2 N^2 reals, interleaved re/im) = rho_c + Z d   (Eq. 6)
    std::vector<double> Z, rho_c;
    double resid_eig = 0, resid_orth = 0;
};

// Check a parameter set. Returns MLN_OK or an error with a message in err.
mln_status validate(const mln_params &p, std::string &err);

// Compute every FP64 constant of the set-up. p must have passed validate().
mln_status build_setup(const mln_params &p, Setup &s, std::string &err);

// Chain rule of the adjoint: from the accumulated gradients of the step's
// constants (acc: A0 - I, b, w, c, T, theta; layout of AccLayout) to the
// gradients of J with respect to the N*N real parameters of mu (diagonal,
// then real and imaginary parts of the upper triangle, row-major) and to the
// relaxation superoperator G (Gamma with dJ = Re sum conj(Gamma_rc) dG_rc).
mln_status adjoint_chain(const mln_params &p, const Setup &s, const double *acc, double *dJ_dmu, double *dJ_dG,
                         std::string &err);

// Stride (in elements) of one adjoint component in the device state.
int64_t state_stride(const mln_params &p);

// Message of the last failed context-free call on this thread (mln_create,
// mln_setup_host, mln_query_buffers, mln_step_noalloc).
std::string &create_error();

}  // namespace mln
