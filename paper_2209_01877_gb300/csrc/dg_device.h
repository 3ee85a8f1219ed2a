// Declarations the kernels' device code depends on: sizes per order, the
// layout of the basis tables, and the arguments of the FP64 / FP32 residual
// kernel.  Host-only declarations live in dg_internal.h.
#pragma once

#include <cstdint>

namespace dg {

// Sizes per polynomial order p (1..3): modes, volume points (symmetric rule
// exact to degree 2p), face points (symmetric triangle rule exact to 2p).
constexpr int nb_of(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }
constexpr int nq_of(int p) { return p == 1 ? 4 : (p == 2 ? 14 : 24); }
constexpr int nqf_of(int p) { return p == 1 ? 3 : (p == 2 ? 6 : 12); }

// Offsets (in elements of the table's scalar type) of the basis tables,
// stored contiguously so a kernel can stage them into shared memory at once:
//   PHIQ  [Nb][Nq]      phi_j at volume point q
//   DPHIW [3][Nq][Nb]   w_q * d phi_j / d xi_k at volume point q
//   PHIF  [4][Nb][Nqf]  phi_j at point q of local face f (own point order)
//   PHIFW [4][Nqf][Nb]  wf_q * phi_j at point q of local face f
//   WQ    [Nq]          volume weights (sum 1/6)
struct TabLayout {
    int nb, nq, nqf;
    int phiq, dphiw, phif, phifw, wq, total;
    explicit TabLayout(int p) {
        nb = nb_of(p); nq = nq_of(p); nqf = nqf_of(p);
        phiq = 0;
        dphiw = phiq + nb * nq;
        phif = dphiw + 3 * nq * nb;
        phifw = phif + 4 * nb * nqf;
        wq = phifw + 4 * nqf * nb;
        total = wq + nq;
    }
};

}  // namespace dg

// Device-side arguments of the residual / RK-stage kernel.
template <typename Real>
struct ResArgs {
    const Real* U;         // residual input [ne][5][Nb] internal order
    const Real* U0;        // RK base state (stages 2, 3)
    Real* out;             // residual or new state
    const int32_t* nbr;    // [ne][4]
    const uint8_t* fcode;  // [ne][4]
    const Real* jinv;      // [ne][9]
    const Real* tab;       // basis tables (TabLayout)
    const int8_t* fperm;   // [6][Nqf]
    int64_t ne;
    Real dt, a, b;         // out = a*U0 + b*(U + dt*R) in RK mode
    Real gamma, roe_eps;
    Real finf[5];          // free-stream conserved state
    const Real* Hs;        // face-once path: per (element, face, point) the face flux, outward
    unsigned int* status;  // device status word
};

