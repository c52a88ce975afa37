// lbm_eos_host.h -- host-side checks and kernel constants of an equation of
// state (Carnahan-Starling, van der Waals Eq. 21, Peng-Robinson Eq. 29),
// shared by every entry point that hands an EOS to a kernel, so that they
// accept the same laws and evaluate them with the same constants.
#pragma once

#include <cmath>

#include "lbm_internal.cuh"

namespace lbm {

// Peng-Robinson alpha(T) = [1 + m (1 - sqrt(T / Tc))]^2 with
// m = 0.37464 + 1.54226 omega - 0.26992 omega^2 (Eq. 29).
inline double pr_alpha(const lbm_eos& e) {
    const double m = 0.37464 + 1.54226 * e.omega - 0.26992 * e.omega * e.omega;
    const double sq = 1.0 + m * (1.0 - std::sqrt(e.T / e.Tc));
    return sq * sq;
}

// A law the kernels can evaluate: a known kind, positive finite constants
// (and a positive critical temperature for Peng-Robinson).  The temperature
// is checked by eos_valid_at().
inline bool eos_valid(const lbm_eos* e) {
    if (!e || (e->kind != LBM_EOS_CS && e->kind != LBM_EOS_VDW && e->kind != LBM_EOS_PR)) return false;
    if (!(e->a > 0) || !(e->b > 0) || !(e->R > 0) || !(e->K > 0) || !std::isfinite(e->a + e->b + e->R + e->K))
        return false;
    if (e->kind == LBM_EOS_PR && (!(e->Tc > 0) || !std::isfinite(e->Tc))) return false;
    return true;
}

// eos_valid() and a positive, finite absolute temperature.
inline bool eos_valid_at(const lbm_eos* e) { return eos_valid(e) && e->T > 0 && std::isfinite(e->T); }

// The EOS members of the kernel constants (K, a, b, b/4, R T, a alpha(T)).
template <typename T> void fill_eos(Phys<T>& P, const lbm_eos& e) {
    P.eos = e.kind;
    P.K = T(e.K);
    P.a = T(e.a);
    P.b = T(e.b);
    P.b4 = T(e.b / 4.0);
    P.RT = T(e.R * e.T);
    P.aalpha = T(e.kind == LBM_EOS_PR ? e.a * pr_alpha(e) : e.a);
}

}  // namespace lbm
