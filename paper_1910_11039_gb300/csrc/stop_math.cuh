// KADABRA stopping functions (arXiv 1910.11039, Section III-A names f and g;
// the formulas are this library's reading):
//   f = (L_L/tau) * (1/3 - omega/tau + sqrt((1/3 - omega/tau)^2 + ((2 b~) omega) / L_L))
//   g = (L_U/tau) * (1/3 + omega/tau + sqrt((1/3 + omega/tau)^2 + ((2 b~) omega) / L_U))
// with b~ = c~(x) / tau and L = -ln(delta).  Written with explicit IEEE
// round-to-nearest intrinsics, which are never contracted into FMAs, so the
// values do not depend on the translation unit's -fmad setting.
#pragma once

namespace kadabra {

// Quantities shared by every vertex of one check.
struct StopConsts {
    double tau_d, omega, af, ag, af2, ag2;
};

__device__ __forceinline__ StopConsts stop_consts(unsigned long long tau, double omega)
{
    StopConsts k;
    k.tau_d = (double)tau;
    k.omega = omega;
    const double r = __ddiv_rn(omega, k.tau_d);
    const double third = 1.0 / 3.0;
    k.af = __dsub_rn(third, r);
    k.ag = __dadd_rn(third, r);
    k.af2 = __dmul_rn(k.af, k.af);
    k.ag2 = __dmul_rn(k.ag, k.ag);
    return k;
}

__device__ __forceinline__ void stop_fg(const StopConsts &k, unsigned int c, double2 L, double &f, double &g)
{
    const double bt = __ddiv_rn((double)c, k.tau_d);
    const double bw = __dmul_rn(__dmul_rn(2.0, bt), k.omega);
    f = __dmul_rn(__ddiv_rn(L.x, k.tau_d), __dadd_rn(k.af, __dsqrt_rn(__dadd_rn(k.af2, __ddiv_rn(bw, L.x)))));
    g = __dmul_rn(__ddiv_rn(L.y, k.tau_d), __dadd_rn(k.ag, __dsqrt_rn(__dadd_rn(k.ag2, __ddiv_rn(bw, L.y)))));
}

// f, g >= +0, so their bit patterns order like the values
__device__ __forceinline__ double fmax_exact(double a, double b) { return b > a ? b : a; }

}  // namespace kadabra
