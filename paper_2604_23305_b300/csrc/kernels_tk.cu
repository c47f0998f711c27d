// Exact pink noise by Timmer & Koenig (1995) over the whole scan (Sect. 2.6, Eq. 20).
//
// For a scan of N samples the plan draws, per (spaxel i, channel ch), the Fourier coefficients of
// a real series of length M = 2^ceil(log2 N) from the one-sided PSD S(f) = A f^-alpha (real and
// imaginary parts of variance M f_s S(f_j) / 4 at f_j = j f_s / M for 0 < j < M/2, a real Nyquist
// coefficient of variance M f_s S / 2, no DC term), inverts the DFT and keeps the first N samples.
// Two channels share one complex inverse FFT: with A_j, B_j Hermitian, the inverse transform of
// A_j + i B_j is a_n + i b_n.  The transform is a Stockham autosort FFT (radix-8 passes and one
// radix-2 or -4 pass, FP32, out of place between two buffers); a tiled transpose then writes the
// series into [n][i][ch], the layout of the TOD, and every run adds its samples to the output.
// All of it runs once, when the plan is prepared; a run costs one elementwise add.
#include <utility>

#include "device_common.cuh"

namespace gateau {
namespace {

constexpr int kTkThreads = 256;

// The normals of Fourier bin j of channel ch come from the Philox draw with counter
// (q lo, q hi, i, 2^30 | ch), q = j >> 1: Box-Muller on words (x, y) for even j, (z, w) for odd j.
// Coefficients X_j / M of the channel pair (2c, 2c + 1) of spaxel i (complex; real at the Nyquist
// bin, zero at DC or for A = 0): sqrt(M f_s A f_j^-alpha / 4) / M = amp_ch f_j^(-alpha/2) with
// amp_ch = sqrt(M f_s A / 4) / M (FP64, once per thread and pair), the power evaluated as
// 2^(-alpha/2 log2 f_j) in FP32 (the FFT runs in FP32 too).  Z[pair][j] = X^a_j + i X^b_j, and
// the conjugate-symmetric half Z[pair][M - j] = conj(X^a_j) + i conj(X^b_j), pair = i P + c.
// A thread takes the two bins j = 2q, 2q + 1 that one Philox draw per channel serves; blocks
// stride over the pairs along y.
__global__ void __launch_bounds__(kTkThreads) tk_spectrum_kernel(float2* __restrict__ Z, int M, int P, int n_pix,
                                                                 int n_ch, const double* __restrict__ A,
                                                                 const double* __restrict__ alpha, double f_sample,
                                                                 uint32_t k0, uint32_t k1) {
    const long long n_pairs = static_cast<long long>(n_pix) * P;
    const float fstep = static_cast<float>(f_sample / M);
    __shared__ float s_amp[2], s_ha[2];
    for (long long pair = blockIdx.y; pair < n_pairs; pair += gridDim.y) {      // uniform over the block
        const int i = static_cast<int>(pair / P), c = static_cast<int>(pair - static_cast<long long>(i) * P);
        // the pair's amplitudes, once per block: FP64 square roots and divisions run at 1/64 of the FP32
        // rate here, and formed by every thread they were most of the kernel
        __syncthreads();
        if (threadIdx.x < 2) {
            const int ch = 2 * c + threadIdx.x;
            const bool live = ch < n_ch && A[ch] > 0.0;
            s_amp[threadIdx.x] = live ? static_cast<float>(sqrt(M * f_sample * A[ch] / 4.0) / M) : 0.f;
            s_ha[threadIdx.x] = live ? -0.5f * static_cast<float>(alpha[ch]) : 0.f;
        }
        __syncthreads();
        float amp[2], ha[2];
        bool on[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            amp[e] = s_amp[e];
            ha[e] = s_ha[e];
            on[e] = amp[e] > 0.f;
        }
        float2* z = Z + pair * M;
        // bins j = 2q, 2q + 1 <= M / 2 < 2^30: 32-bit indices (a 64-bit integer's conversion to float
        // runs on the FP64 pipe, which it had kept ~70 % busy)
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; 2 * q <= M / 2; q += gridDim.x * blockDim.x) {
            uint4 x[2];
#pragma unroll
            for (int e = 0; e < 2; ++e)
                x[e] = philox4x32_10(make_uint4(static_cast<uint32_t>(q), 0u, static_cast<uint32_t>(i),
                                                0x40000000u | static_cast<uint32_t>(2 * c + e)),
                                     k0, k1);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = 2 * q + h;
                if (j > M / 2) break;
                const float lf = j > 0 ? log2f(static_cast<float>(j) * fstep) : 0.f;
                float2 cf[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    if (!on[e] || j == 0) {
                        cf[e] = make_float2(0.f, 0.f);
                        continue;
                    }
                    const float a = amp[e] * exp2f(ha[e] * lf);
                    const float2 n = h ? box_muller(x[e].z, x[e].w) : box_muller(x[e].x, x[e].y);
                    cf[e] = 2 * j == M ? make_float2(1.41421356237f * a * n.x, 0.f)   // real Nyquist coefficient
                                       : make_float2(a * n.x, a * n.y);
                }
                z[j] = make_float2(cf[0].x - cf[1].y, cf[0].y + cf[1].x);
                if (j > 0 && 2 * j < M) z[M - j] = make_float2(cf[0].x + cf[1].y, cf[1].x - cf[0].y);
            }
        }
    }
}

// One Stockham pass over rows of length M: sub-transforms of length Ns become length R Ns.
// SIGN = +1: e^{+2 pi i jk/M} (inverse, unscaled); -1: e^{-2 pi i jk/M} (forward).
template <int R, int SIGN>
__global__ void __launch_bounds__(kTkThreads) stockham_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                                              int M, int Ns, long long n_pairs) {
    const int MR = M / R;
    const long long total = n_pairs * MR;
    for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long pair = t / MR;
        const int j = static_cast<int>(t - pair * MR);
        const float2* src = in + pair * M;
        float2* dst = out + pair * M;
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 x = src[j + r * MR];
            // twiddle e^{+2 pi i r k / (R Ns)}: (r k) mod (R Ns) and the power-of-two divisor are exact
            float s, c;
            sincospif(2.0f * static_cast<float>((r * k) % (R * Ns)) / static_cast<float>(R * Ns), &s, &c);
            s *= SIGN;
            v[r] = make_float2(x.x * c - x.y * s, x.x * s + x.y * c);
        }
        const int idx = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float s, c;
                sincospif(2.0f * static_cast<float>((r * q) % R) / static_cast<float>(R), &s, &c);   // constants
                s *= SIGN;
                acc.x += v[r].x * c - v[r].y * s;
                acc.y += v[r].x * s + v[r].y * c;
            }
            dst[idx + q * Ns] = acc;
        }
    }
}

// tk[n][i][ch] = scale[ch] * (Re or Im of Z[i P + ch/2][n]) for n < N: 32 x 32 tiles through shared memory.
__global__ void __launch_bounds__(256) tk_scatter_kernel(const float2* __restrict__ Z, int M, int P, int n_pix, int n_ch,
                                                         long long N, const float* __restrict__ scale,
                                                         float* __restrict__ tk) {
    __shared__ float tile[32][33];
    const long long S = static_cast<long long>(n_pix) * n_ch;
    const long long n0 = static_cast<long long>(blockIdx.x) * 32;
    const long long s0 = static_cast<long long>(blockIdx.y) * 32;
    for (int sl = threadIdx.y; sl < 32; sl += 8) {
        const long long s = s0 + sl, n = n0 + threadIdx.x;
        float v = 0.f;
        if (s < S && n < N) {
            const int i = static_cast<int>(s / n_ch), ch = static_cast<int>(s - static_cast<long long>(i) * n_ch);
            const float2 z = Z[(static_cast<long long>(i) * P + (ch >> 1)) * M + n];
            v = (ch & 1) ? z.y : z.x;
        }
        tile[sl][threadIdx.x] = v;
    }
    __syncthreads();
    for (int nl = threadIdx.y; nl < 32; nl += 8) {
        const long long n = n0 + nl, s = s0 + threadIdx.x;
        if (s < S && n < N) {
            const int ch = static_cast<int>(s % n_ch);
            tk[n * S + s] = tile[threadIdx.x][nl] * (scale ? scale[ch] : 1.f);
        }
    }
}

__global__ void __launch_bounds__(256) tk_add_kernel(float* __restrict__ out, const float* __restrict__ tk, long long count) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < count;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        out[e] += tk[e];
}

int grid_for(long long work, int threads) {
    const long long b = (work + threads - 1) / threads;
    return static_cast<int>(b < 148LL * 32 ? (b > 0 ? b : 1) : 148LL * 32);
}

}  // namespace

long long tk_length(long long n_total) {
    long long M = 2;
    while (M < n_total) M <<= 1;
    return M;
}

cudaError_t launch_tk_realise(const double* A, const double* alpha, double f_sample, uint32_t k0, uint32_t k1, int n_pix,
                              int n_ch, long long n_total, const float* scale, float2* work0, float2* work1, float* tk,
                              cudaStream_t stream) {
    const long long M = tk_length(n_total);
    if (M > (1LL << 30) || n_ch < 1 || n_pix < 1) return cudaErrorInvalidValue;
    const int P = (n_ch + 1) / 2;
    const long long n_pairs = static_cast<long long>(n_pix) * P;
    const long long nq = M / 4 + 1;                  // thread items per pair (bins 2q, 2q + 1)
    const dim3 sgrid(static_cast<unsigned>((nq + kTkThreads - 1) / kTkThreads < 64 ? (nq + kTkThreads - 1) / kTkThreads : 64),
                     static_cast<unsigned>(n_pairs < 65535 ? n_pairs : 65535));
    tk_spectrum_kernel<<<sgrid, kTkThreads, 0, stream>>>(work0, static_cast<int>(M), P, n_pix, n_ch, A, alpha,
                                                         f_sample, k0, k1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const float2* in = nullptr;
    e = launch_fft_rows(work0, work1, n_pairs, static_cast<int>(M), +1, &in, stream);
    if (e != cudaSuccess) return e;
    const long long S = static_cast<long long>(n_pix) * n_ch;
    const dim3 grid(static_cast<unsigned>((n_total + 31) / 32), static_cast<unsigned>((S + 31) / 32));
    if (grid.y > 65535u) return cudaErrorInvalidValue;
    tk_scatter_kernel<<<grid, dim3(32, 8), 0, stream>>>(in, static_cast<int>(M), P, n_pix, n_ch, n_total, scale, tk);
    return cudaGetLastError();
}

template <int SIGN>
cudaError_t fft_rows_dir(float2* a, float2* b, long long rows, int M, const float2** result, cudaStream_t stream) {
    int p = 0;
    while ((1 << p) < M) ++p;
    float2* in = a;
    float2* out = b;
    int Ns = 1;
    for (int q = 0; q < p / 3; ++q) {
        stockham_kernel<8, SIGN><<<grid_for(rows * (M / 8), kTkThreads), kTkThreads, 0, stream>>>(in, out, M, Ns, rows);
        Ns *= 8;
        std::swap(in, out);
    }
    if (p % 3 == 1) {
        stockham_kernel<2, SIGN><<<grid_for(rows * (M / 2), kTkThreads), kTkThreads, 0, stream>>>(in, out, M, Ns, rows);
        std::swap(in, out);
    } else if (p % 3 == 2) {
        stockham_kernel<4, SIGN><<<grid_for(rows * (M / 4), kTkThreads), kTkThreads, 0, stream>>>(in, out, M, Ns, rows);
        std::swap(in, out);
    }
    *result = in;
    return cudaGetLastError();
}

cudaError_t launch_fft_rows(float2* a, float2* b, long long rows, int M, int sign, const float2** result,
                            cudaStream_t stream) {
    if (M < 2 || (M & (M - 1)) != 0 || rows < 1) return cudaErrorInvalidValue;
    return sign > 0 ? fft_rows_dir<+1>(a, b, rows, M, result, stream) : fft_rows_dir<-1>(a, b, rows, M, result, stream);
}

cudaError_t launch_tk_add(float* out, const float* tk, long long count, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    tk_add_kernel<<<grid_for(count, 256), 256, 0, stream>>>(out, tk, count);
    return cudaGetLastError();
}

}  // namespace gateau
