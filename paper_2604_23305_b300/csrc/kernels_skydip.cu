// Brightness-temperature scale by a simulated skydip (Sect. 2.7).
//
// The zenith PWV is swept over n_dip values at the scan's base elevation with no source; for
// each value and channel the kernel forms, in FP64,
//   P_KID = sum_nu eta_filt w [c0 + c1 (1 - eta_atm)]          (Eq. 16 on the collapsed cascade)
//   T_b   = T_atm sum_nu eta_filt w (1 - eta_atm) / sum_nu eta_filt w
// with eta_atm = exp(-csc(el) tau_z(PWV, nu)) (Eq. 10) and tau_z interpolated linearly between
// the rows of the plan's opacity table (PWV clamped to the table), then fits the least-squares
// line T_b = a P_KID + b.  One block per channel; it runs once when the plan is prepared.
#include "gateau_internal.h"

namespace gateau {
namespace {

constexpr int kSkydipThreads = 256;

__device__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();                      // red[] free from the previous call
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < (kSkydipThreads / 32) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;                             // valid in thread 0
}

__global__ void __launch_bounds__(kSkydipThreads) skydip_fit_kernel(
    const double* __restrict__ hw, const double* __restrict__ c01, const float* __restrict__ tau, int n_freq, int Kp,
    int n_pwv, double pwv_min, double dpwv, double csc_el, double T_atm, double pwv_lo, double pwv_hi, int n_dip,
    int n_ch, double* __restrict__ ab, float* __restrict__ ab_f, int ab_f_stride) {
    __shared__ double red[kSkydipThreads / 32];
    __shared__ double Pm[kMaxSkydip], Tm[kMaxSkydip];
    const int ch = blockIdx.x;
    const double* h = hw + static_cast<size_t>(ch) * n_freq;
    double sh = 0.0;
    for (int k = threadIdx.x; k < n_freq; k += kSkydipThreads) sh += h[k];
    const double SH = block_sum(sh, red);
    for (int m = 0; m < n_dip; ++m) {
        const double pwv = pwv_lo + (pwv_hi - pwv_lo) * m / (n_dip - 1);
        double u = (pwv - pwv_min) / dpwv;
        u = fmin(fmax(u, 0.0), static_cast<double>(n_pwv - 1));
        const int j = min(static_cast<int>(floor(u)), n_pwv - 2);
        const double f = u - j;
        const float* t0 = tau + static_cast<size_t>(2 * j) * Kp;      // tau_j
        const float* dt = t0 + Kp;                                     // tau_{j+1} - tau_j
        double sp = 0.0, st = 0.0;
        for (int k = threadIdx.x; k < n_freq; k += kSkydipThreads) {
            const double tz = static_cast<double>(t0[k]) + f * static_cast<double>(dt[k]);
            const double one_minus_eta = -expm1(-csc_el * tz);
            sp += h[k] * (c01[k] + c01[n_freq + k] * one_minus_eta);
            st += h[k] * one_minus_eta;
        }
        const double P = block_sum(sp, red);
        const double S = block_sum(st, red);
        if (threadIdx.x == 0) {
            Pm[m] = P;
            Tm[m] = SH > 0.0 ? T_atm * S / SH : 0.0;
        }
    }
    if (threadIdx.x == 0) {
        double mp = 0.0, mt = 0.0;
        for (int m = 0; m < n_dip; ++m) {
            mp += Pm[m];
            mt += Tm[m];
        }
        mp /= n_dip;
        mt /= n_dip;
        double sxy = 0.0, sxx = 0.0;
        for (int m = 0; m < n_dip; ++m) {
            sxy += (Pm[m] - mp) * (Tm[m] - mt);
            sxx += (Pm[m] - mp) * (Pm[m] - mp);
        }
        // a channel that sees no sky change (no band, or an opaque / transparent sweep) keeps a = 0
        const double a = sxx > 0.0 ? sxy / sxx : 0.0;
        const double b = mt - a * mp;
        ab[ch] = a;
        ab[n_ch + ch] = b;
        ab_f[ch] = static_cast<float>(a);
        ab_f[ab_f_stride + ch] = static_cast<float>(b);
    }
}

}  // namespace

cudaError_t launch_skydip_fit(const double* hw, const double* c01, const float* tau, int n_freq, int Kp, int n_pwv,
                              double pwv_min, double dpwv, double csc_el, double T_atm, double pwv_lo, double pwv_hi,
                              int n_dip, int n_ch, double* ab, float* ab_f, int ab_f_stride, cudaStream_t stream) {
    if (n_dip < 2 || n_dip > kMaxSkydip || n_ch < 1 || n_pwv < 2) return cudaErrorInvalidValue;
    skydip_fit_kernel<<<n_ch, kSkydipThreads, 0, stream>>>(hw, c01, tau, n_freq, Kp, n_pwv, pwv_min, dpwv, csc_el,
                                                           T_atm, pwv_lo, pwv_hi, n_dip, n_ch, ab, ab_f, ab_f_stride);
    return cudaGetLastError();
}

}  // namespace gateau
