// Downstream of the TOD: the common-mode reduction of Sect. 4.3 (Eqs. 25-26).
//
// For a brightness-temperature TOD T_b[t][i][ch] each (sample, channel) column is reduced over
// the spaxels that see no source (S_j = 1, Eq. 26) to the common atmosphere term
//   C = (1 / N_out) sum_j S_j T_b,j / (1 - eta_j),
// and every spaxel gets T*_a,i = T_b,i / eta_i - (1 - eta_i) / eta_i * C (Eq. 25), with
// eta_i = eta_z^csc(el_i(t)) (Eq. 10) from the band transmission eta_z of the channel at the
// observation's mean zenith PWV.  The elevations come from the row-setup kernel (RowParams.csc),
// and so do the line-of-sight PWVs that the mean zenith PWV averages.
#include "gateau_internal.h"

namespace gateau {
namespace {

constexpr int kReduceThreads = 256;

__global__ void __launch_bounds__(kReduceThreads) sum_pwv_kernel(const RowParams* __restrict__ rows, long long n,
                                                                 double* __restrict__ sum) {
    __shared__ double red[kReduceThreads / 32];
    double s = 0.0;
    for (long long r = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; r < n;
         r += static_cast<long long>(gridDim.x) * blockDim.x)
        s += static_cast<double>(rows[r].pwv);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < kReduceThreads / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(sum, s);
    }
}

// log eta_z of each channel: eta_z = sum_nu eta_filt w exp(-tau_z(PWV, nu)) / sum_nu eta_filt w, with
// tau_z interpolated between the opacity-table rows as everywhere else (PWV clamped to the table).
__global__ void __launch_bounds__(kReduceThreads) band_transmission_kernel(
    const double* __restrict__ hw, const float* __restrict__ tau, int n_freq, int Kp, int n_pwv, double pwv_min,
    double dpwv, double pwv, float* __restrict__ log_eta_z) {
    __shared__ double red[2][kReduceThreads / 32];
    const double* h = hw + static_cast<size_t>(blockIdx.x) * n_freq;
    double u = (pwv - pwv_min) / dpwv;
    u = fmin(fmax(u, 0.0), static_cast<double>(n_pwv - 1));
    const int j = min(static_cast<int>(floor(u)), n_pwv - 2);
    const double f = u - j;
    const float* t0 = tau + static_cast<size_t>(2 * j) * Kp;
    const float* dt = t0 + Kp;
    double se = 0.0, sh = 0.0;
    for (int k = threadIdx.x; k < n_freq; k += kReduceThreads) {
        se += h[k] * exp(-(static_cast<double>(t0[k]) + f * static_cast<double>(dt[k])));
        sh += h[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        se += __shfl_down_sync(0xffffffffu, se, o);
        sh += __shfl_down_sync(0xffffffffu, sh, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = se;
        red[1][threadIdx.x >> 5] = sh;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kReduceThreads / 32; ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        log_eta_z[blockIdx.x] = b > 0.0 ? static_cast<float>(log(a / b)) : 0.f;
    }
}

// One thread per (sample, channel) column; out may be tb (each column is read before it is written).
__global__ void __launch_bounds__(kReduceThreads) common_mode_kernel(const float* tb, float* out,
                                                                     const RowParams* __restrict__ rows, long long nt,
                                                                     int n_pix, int n_ch,
                                                                     const float* __restrict__ log_eta_z,
                                                                     const unsigned char* __restrict__ off_source,
                                                                     float inv_n_out) {
    const long long cols = nt * n_ch;
    for (long long c = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; c < cols;
         c += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long t = c / n_ch;
        const int ch = static_cast<int>(c - t * n_ch);
        const float lz = log_eta_z[ch];
        const long long base = t * n_pix * static_cast<long long>(n_ch) + ch;
        float common = 0.f;
        for (int j = 0; j < n_pix; ++j) {
            if (!off_source[j]) continue;
            const float a = rows[static_cast<long long>(j) * nt + t].csc * lz;     // ln eta_j
            common += tb[base + static_cast<long long>(j) * n_ch] / -expm1f(a);   // T_b,j / (1 - eta_j)
        }
        common *= inv_n_out;
        for (int i = 0; i < n_pix; ++i) {
            const float a = rows[static_cast<long long>(i) * nt + t].csc * lz;
            const long long e = base + static_cast<long long>(i) * n_ch;
            out[e] = (tb[e] + expm1f(a) * common) * expf(-a);                     // Eq. 25
        }
    }
}

// e^a on the special-function unit (relative error ~2^-22).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// e^a - 1 for a <= 0 (a = csc ln eta_z): the Taylor series to a^7 where cancellation would cost
// digits (|a| < 1/4: truncation < 3e-9 relative), 2^(a log2 e) - 1 beyond (|e^a - 1| > 0.22 there).
__device__ __forceinline__ float expm1_neg(float a) {
    if (a > -0.25f)
        return a * (1.f + a * (0.5f + a * (1.f / 6 + a * (1.f / 24 + a * (1.f / 120 + a * (1.f / 720 + a * (1.f / 5040)))))));
    return ex2_approx(a * 1.4426950408889634f) - 1.f;
}

// A whole sample (all spaxels and channels, n_pix n_ch floats) per block in shared memory: the TOD
// is read and written with unit stride, and each channel's column is reduced from shared memory.
constexpr int kTileMaxFloats = 12 * 1024;          // 48 KB of slab (+ the spaxels' csc)
__global__ void __launch_bounds__(kReduceThreads) common_mode_tile_kernel(const float* tb, float* out,
                                                                          const RowParams* __restrict__ rows,
                                                                          long long nt, int n_pix, int n_ch,
                                                                          const float* __restrict__ log_eta_z,
                                                                          const unsigned char* __restrict__ off_source,
                                                                          float inv_n_out) {
    extern __shared__ float slab[];                 // [n_pix][n_ch], then csc [n_pix]
    const int S = n_pix * n_ch;
    float* csc = slab + S;
    for (long long t = blockIdx.x; t < nt; t += gridDim.x) {
        const float* src = tb + t * S;
        // eight loads in flight per thread before their shared-memory stores
        for (int e0 = threadIdx.x; e0 < S; e0 += 8 * kReduceThreads) {
            float r[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * kReduceThreads;
                r[u] = e < S ? src[e] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * kReduceThreads;
                if (e < S) slab[e] = r[u];
            }
        }
        for (int j = threadIdx.x; j < n_pix; j += blockDim.x) csc[j] = rows[static_cast<long long>(j) * nt + t].csc;
        __syncthreads();
        for (int ch = threadIdx.x; ch < n_ch; ch += blockDim.x) {
            const float lz = log_eta_z[ch];
            float common = 0.f;
            for (int j = 0; j < n_pix; ++j)
                if (off_source[j]) common += __fdividef(slab[j * n_ch + ch], -expm1_neg(csc[j] * lz));   // T_b,j / (1 - eta_j)
            common *= inv_n_out;
            for (int i = 0; i < n_pix; ++i) {
                const float a = csc[i] * lz;                                            // ln eta_i
                slab[i * n_ch + ch] = (slab[i * n_ch + ch] + expm1_neg(a) * common) * ex2_approx(-a * 1.4426950408889634f);
            }
        }
        __syncthreads();
        float* dst = out + t * S;
        for (int e = threadIdx.x; e < S; e += blockDim.x) dst[e] = slab[e];
        __syncthreads();
    }
}

int grid_for(long long work) {
    const long long b = (work + kReduceThreads - 1) / kReduceThreads;
    return static_cast<int>(b < 148LL * 16 ? (b > 0 ? b : 1) : 148LL * 16);
}

}  // namespace

cudaError_t launch_sum_pwv(const RowParams* rows, long long n, double* sum, cudaStream_t stream) {
    sum_pwv_kernel<<<grid_for(n), kReduceThreads, 0, stream>>>(rows, n, sum);
    return cudaGetLastError();
}

cudaError_t launch_band_transmission(const double* hw, const float* tau, int n_freq, int Kp, int n_pwv, double pwv_min,
                                     double dpwv, double pwv, int n_ch, float* log_eta_z, cudaStream_t stream) {
    band_transmission_kernel<<<n_ch, kReduceThreads, 0, stream>>>(hw, tau, n_freq, Kp, n_pwv, pwv_min, dpwv, pwv,
                                                                  log_eta_z);
    return cudaGetLastError();
}

cudaError_t launch_common_mode(const float* tb, float* out, const RowParams* rows, long long nt, int n_pix, int n_ch,
                               const float* log_eta_z, const unsigned char* off_source, int n_out,
                               cudaStream_t stream) {
    if (n_out < 1) return cudaErrorInvalidValue;
    if (static_cast<long long>(n_pix) * n_ch <= kTileMaxFloats) {
        const size_t smem = (static_cast<size_t>(n_pix) * n_ch + n_pix) * sizeof(float);
        const long long blocks = nt < 148LL * 6 ? nt : 148LL * 6;
        common_mode_tile_kernel<<<static_cast<unsigned>(blocks), kReduceThreads, smem, stream>>>(
            tb, out, rows, nt, n_pix, n_ch, log_eta_z, off_source, 1.0f / static_cast<float>(n_out));
    } else
        common_mode_kernel<<<grid_for(nt * n_ch), kReduceThreads, 0, stream>>>(
            tb, out, rows, nt, n_pix, n_ch, log_eta_z, off_source, 1.0f / static_cast<float>(n_out));
    return cudaGetLastError();
}

}  // namespace gateau
