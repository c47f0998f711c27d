// Preprocessing on the device (Sect. 2.2, Eqs. 1-3): the telescope far field, the beam convolution
// of the source cube and the footprint smoothing of the PWV screen.
//
// Aperture illumination (Eq. 2): a Gaussian whose amplitude falls to t_edge dB at the rim,
// A(r) = 10^((t_edge/20) (r/R)^2) for r < R, 0 outside, sampled in wavelengths (l, m) with spacings
// 1/(N_a pitch_az), 1/(N_e pitch_el) so that its 2-D DFT lands on the angular grid of the cube
// (offset q pitch at index q mod N).  F = |DFT A|^2, normalised to a peak of 1 (Eq. 3).  Eq. 1 is
// the linear convolution of I cos(el') with F on the cube's grid times A_p dphi dtheta, done as a
// product of transforms on grids of twice the cube's size.  Every 2-D transform is two passes of
// the batched row FFT with a tiled transpose after each.  Frequencies go through in batches.
#include <mutex>
#include <set>
#include <utility>

#include "gateau_internal.h"

namespace gateau {
namespace {

constexpr int kPrepThreads = 256;
constexpr double kC = 299792458.0;

int grid_for(long long work) {
    const long long b = (work + kPrepThreads - 1) / kPrepThreads;
    return static_cast<int>(b < 148LL * 32 ? (b > 0 ? b : 1) : 148LL * 32);
}

__device__ __forceinline__ double fft_offset(int q, int n) { return q < n / 2 ? q : q - n; }

__device__ __forceinline__ double illumination(double r, double R, double t_edge_db) {
    return r < R ? exp10((t_edge_db / 20.0) * (r / R) * (r / R)) : 0.0;
}

// A_b(l_q, m_p) for plane b = frequency nu[b].
__global__ void aperture_kernel(float2* __restrict__ A, const double* __restrict__ nu, int na, int ne, float inv_laz,
                                float inv_lel, double R, float t_edge_20) {
    // plane b = blockIdx.y; its wavelength over the aperture radius formed once per block (FP64
    // divisions run at 1/64 of the FP32 rate on this part: once per thread they were most of the
    // kernel), the direction cosines in FP32 (the plane is FP32, and l, m stay far below float's limits)
    const int b = blockIdx.y;
    __shared__ float s_lam_R;
    if (threadIdx.x == 0) s_lam_R = static_cast<float>(kC / nu[b] / R);
    __syncthreads();
    const float lam_R = s_lam_R;
    const int plane = na * ne;                       // <= 4096 x 4096: 32-bit indices within a plane
    float2* Ab = A + static_cast<long long>(b) * plane;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < plane; t += gridDim.x * blockDim.x) {
        const int q = t / ne, p = t - q * ne;
        const float l = static_cast<float>(q < na / 2 ? q : q - na) * inv_laz;
        const float m = static_cast<float>(p < ne / 2 ? p : p - ne) * inv_lel;
        const float rr = lam_R * hypotf(l, m);
        Ab[t] = make_float2(rr < 1.f ? exp10f(t_edge_20 * rr * rr) : 0.f, 0.f);
    }
}

// [B][n0][n1] -> [B][n1][n0], 32 x 32 tiles.
__global__ void transpose_kernel(const float2* __restrict__ in, float2* __restrict__ out, int n0, int n1) {
    __shared__ float2 tile[32][33];
    const size_t plane = static_cast<size_t>(n0) * n1;
    const float2* src = in + blockIdx.z * plane;
    float2* dst = out + blockIdx.z * plane;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;      // tile of columns (n1) and rows (n0)
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        if (r < n0 && c < n1) tile[y][threadIdx.x] = src[static_cast<size_t>(r) * n1 + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (r < n0 && c < n1) dst[static_cast<size_t>(c) * n0 + r] = tile[threadIdx.x][y];
    }
}

// |E|^2 per plane and its maximum (one block per plane).
// |E|^2 in place and its maximum per plane: blockIdx.y = plane, blockIdx.x strides over it; the
// maximum is combined with an integer atomic max on the bits of the (non-negative) floats, so
// peak must be zero on entry.
__global__ void power_max_kernel(float2* __restrict__ E, long long plane, float* __restrict__ peak) {
    __shared__ float red[kPrepThreads / 32];
    float2* e = E + blockIdx.y * plane;
    float mx = 0.f;
    for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < plane;
         t += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float2 v = e[t];
        const float pw = v.x * v.x + v.y * v.y;
        e[t] = make_float2(pw, 0.f);
        mx = fmaxf(mx, pw);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < kPrepThreads / 32; ++w) m = fmaxf(m, red[w]);
        atomicMax(reinterpret_cast<int*>(peak) + blockIdx.y, __float_as_int(m));
    }
}

// E /= its plane's maximum: blockIdx.y = plane, blockIdx.x strides over it.
__global__ void scale_planes_kernel(float2* __restrict__ E, long long plane, const float* __restrict__ peak) {
    float2* e = E + blockIdx.y * plane;
    const float s = 1.f / peak[blockIdx.y];
    for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < plane;
         t += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float2 v = e[t];
        e[t] = make_float2(v.x * s, v.y * s);
    }
}

// Source planes: S[b][a][e] = I[a][e][f0 + b] cos(el0 + e d_el) inside the cube, 0 in the padding.
// The cube runs along frequency and the planes along elevation, so a block moves a 32 (elevation)
// x 32 (frequency) tile of row a through shared memory: both the reads and the writes are coalesced.
// grid (padded elevation / 32, frequencies of the batch / 32, padded azimuth), block 32 x 8.
__global__ void source_planes_kernel(const float* __restrict__ I, float2* __restrict__ S, int B, int f0, int n_freq,
                                     int n_az, int n_el, double el0, double d_el) {
    __shared__ float tile[32][33];                   // [elevation][frequency]
    const int na = 2 * n_az, ne = 2 * n_el;
    const int e0 = blockIdx.x * 32, b0 = blockIdx.y * 32, a = blockIdx.z;
    const bool in_cube = a < n_az;
    if (in_cube) {
        for (int y = threadIdx.y; y < 32; y += 8) {
            const int e = e0 + y, b = b0 + threadIdx.x;
            float v = 0.f;
            if (e < n_el && b < B)
                v = I[(static_cast<size_t>(a) * n_el + e) * n_freq + f0 + b] * cosf(static_cast<float>(el0 + e * d_el));
            tile[y][threadIdx.x] = v;
        }
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int b = b0 + y, e = e0 + threadIdx.x;
        if (b < B && e < ne)
            S[(static_cast<size_t>(b) * na + a) * ne + e] = make_float2(in_cube && e < n_el ? tile[threadIdx.x][y] : 0.f, 0.f);
    }
}

// S *= K / peak of its plane (the beam's normalisation, applied here: its transform is linear):
// blockIdx.y = plane, blockIdx.x strides over it.
__global__ void multiply_scaled_kernel(float2* __restrict__ S, const float2* __restrict__ K, long long plane,
                                       const float* __restrict__ peak) {
    float2* s = S + blockIdx.y * plane;
    const float2* k = K + blockIdx.y * plane;
    const float r = 1.f / peak[blockIdx.y];
    for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < plane;
         t += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float2 a = s[t], kb = k[t];
        const float2 b = make_float2(kb.x * r, kb.y * r);
        s[t] = make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
    }
}

__global__ void multiply_kernel(float2* __restrict__ S, const float2* __restrict__ K, long long n) {
    for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < n;
         t += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float2 a = S[t], b = K[t];
        S[t] = make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
    }
}

// P[a][e][f0 + b] = scale Re S[b][a][e] for the cube's cells, through 32 (elevation) x 32
// (frequency) tiles of row a in shared memory (coalesced on both sides).
// grid (n_el / 32, frequencies of the batch / 32, n_az), block 32 x 8.
__global__ void gather_planes_kernel(const float2* __restrict__ S, float* __restrict__ P, int B, int f0, int n_freq,
                                     int n_az, int n_el, float scale) {
    __shared__ float tile[32][33];                   // [frequency][elevation]
    const int ne = 2 * n_el;
    const long long plane = static_cast<long long>(2 * n_az) * ne;
    const int e0 = blockIdx.x * 32, b0 = blockIdx.y * 32, a = blockIdx.z;
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int b = b0 + y, e = e0 + threadIdx.x;
        tile[y][threadIdx.x] = (b < B && e < n_el) ? S[b * plane + static_cast<long long>(a) * ne + e].x : 0.f;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int e = e0 + y, b = b0 + threadIdx.x;
        if (e < n_el && b < B) P[(static_cast<size_t>(a) * n_el + e) * n_freq + f0 + b] = scale * tile[threadIdx.x][y];
    }
}

// Footprint of the screen smoothing: A(r) on the screen grid in metres (offsets in DFT order) and its sum.
__global__ void footprint_kernel(float2* __restrict__ K, int nx, int ny, double pitch, double R, double t_edge_db,
                                 double* __restrict__ sum) {
    __shared__ double red[kPrepThreads / 32];
    const long long total = static_cast<long long>(nx) * ny;
    double s = 0.0;
    for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int y = static_cast<int>(t / nx), x = static_cast<int>(t - static_cast<long long>(y) * nx);
        const double v = illumination(pitch * hypot(fft_offset(x, nx), fft_offset(y, ny)), R, t_edge_db);
        K[t] = make_float2(static_cast<float>(v), 0.f);
        s += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < kPrepThreads / 32; ++w) a += red[w];
        atomicAdd(sum, a);
    }
}

__global__ void to_complex_kernel(const float* __restrict__ in, float2* __restrict__ out, long long n) {
    for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < n;
         t += static_cast<long long>(gridDim.x) * blockDim.x)
        out[t] = make_float2(in[t], 0.f);
}

// out = Re(in) * scale[0 or by the FP64 divisor]: scale_by is null or a device double (1 / (n scale_by)).
__global__ void real_part_kernel(const float2* __restrict__ in, float* __restrict__ out, long long n, double scale,
                                 const double* __restrict__ divisor) {
    const double s = divisor ? scale / divisor[0] : scale;
    for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < n;
         t += static_cast<long long>(gridDim.x) * blockDim.x)
        out[t] = static_cast<float>(in[t].x * s);
}

}  // namespace

cudaError_t launch_real_part(const float2* in, float* out, long long n, cudaStream_t stream) {
    real_part_kernel<<<grid_for(n), kPrepThreads, 0, stream>>>(in, out, n, 1.0, nullptr);
    return cudaGetLastError();
}

// 2-D transform of B planes [n0][n1] held in a (b is scratch); the result is left in a.
// One-pass transforms of whole vectors in shared memory: a block takes V vectors of n points
// (V n <= 4096 complex values), loads them in bit-reversed order, runs the log2 n
// decimation-in-time stages in place (pairs of stages fused into radix-4 butterflies), and stores
// them back in place.  Vector v starts at (v / per_plane) * plane_stride + (v % per_plane) * vstride
// and its points are kstride apart: rows of a plane (kstride 1, contiguous) or its columns
// (kstride = row length; a block's V columns are adjacent, so each point's loads are coalesced).
// n, V and per_plane are powers of two, passed as their logarithms: every index is a shift or a mask.
//
// Shared-memory layout.  A bank row holds 16 complex values, and a half-warp's 8-byte accesses are
// conflict-free when they fall in 16 distinct slots (index mod 16).  The bit-reversed scatter, the
// column loads (16 vectors at one point) and the early radix-4 stages (strides 1, 4, 16 in a
// vector) would each put a half-warp on one or a few slots, so point k of vector vl is held at
//   vl (n + 1) + swz(k),   swz(k) = k ^ (((k >> 4) * 5 ^ (k >> 8)) & 15):
// the odd vector stride spreads adjacent vectors over the slots, and the XOR (a permutation of the
// 16 slots of each bank row, chosen by its row index) spreads strided points; an exhaustive count
// over every access pattern of the kernel gives no conflict for n = 64, 128, 256 and 4096 and at
// most two-way for the other sides.  The twiddles sit after the data as one table per stage size,
// tw[h + p] = e^{sign pi i p / h} (h a power of two, p < h), which a half-warp reads contiguously.
constexpr int kFftSmemPoints = 4096;            // V n <= this many complex values per block
__device__ __forceinline__ int fft_swz(int k) { return k ^ ((((k >> 4) * 5) ^ (k >> 8)) & 15); }

size_t fft_smem_bytes(int n, int V) { return (static_cast<size_t>(V) * (n + 1) + n) * sizeof(float2); }

template <int SIGN>
__global__ void __launch_bounds__(kPrepThreads) fft_smem_kernel(float2* a, long long nvec, int log2n, long long kstride,
                                                                 int log2pp, long long vstride, long long plane_stride,
                                                                 int log2V) {
    const int n = 1 << log2n, V = 1 << log2V;
    const int sv = n + 1;                        // vector stride in shared memory
    extern __shared__ float2 sm[];
    float2* tw = sm + V * sv;                    // tw[h + p] = e^{sign pi i p / h}, 1 <= h + p < n
    const bool columns = kstride != 1;
    const int nv = V * n;
    for (int m = 1 + threadIdx.x; m < n; m += blockDim.x) {
        const int lh = 31 - __clz(m);
        float sn, cs;
        sincospif(static_cast<float>(m - (1 << lh)) / static_cast<float>(1 << lh), &sn, &cs);   // exact divisor
        tw[m] = make_float2(cs, SIGN * sn);
    }
    const long long pp_mask = (1LL << log2pp) - 1;
    for (long long v0 = static_cast<long long>(blockIdx.x) * V; v0 < nvec; v0 += static_cast<long long>(gridDim.x) * V) {
        auto base = [&](long long v) { return (v >> log2pp) * plane_stride + (v & pp_mask) * vstride; };
        for (int t = threadIdx.x; t < nv; t += blockDim.x) {
            // columns: the block's V vectors vary fastest (adjacent addresses); rows: the points do
            const int vl = columns ? (t & (V - 1)) : (t >> log2n), k = columns ? (t >> log2V) : (t & (n - 1));
            const long long v = v0 + vl;
            const int kr = static_cast<int>(__brev(static_cast<unsigned>(k)) >> (32 - log2n));
            sm[vl * sv + fft_swz(kr)] = v < nvec ? a[base(v) + k * kstride] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        // stages of half-size 2^lh; an odd count starts with one radix-2 stage, the rest go in
        // fused pairs (half-sizes h, 2h: one radix-4 butterfly, one shared-memory round trip)
        int lh = 0;
        if (log2n & 1) {
            for (int t = threadIdx.x; t < nv / 2; t += blockDim.x) {
                const int vl = t >> (log2n - 1), j = t & (n / 2 - 1);
                const int i0 = vl * sv + fft_swz(2 * j), i1 = vl * sv + fft_swz(2 * j + 1);   // half 1: twiddle 1
                const float2 u = sm[i0], w = sm[i1];
                sm[i0] = make_float2(u.x + w.x, u.y + w.y);
                sm[i1] = make_float2(u.x - w.x, u.y - w.y);
            }
            __syncthreads();
            lh = 1;
        }
        for (; lh < log2n; lh += 2) {
            const int h = 1 << lh;
            for (int t = threadIdx.x; t < nv / 4; t += blockDim.x) {
                const int vl = t >> (log2n - 2), j = t & (n / 4 - 1);
                const int pos = j & (h - 1), grp = j >> lh;
                const int k0 = (grp << (lh + 2)) + pos, vb = vl * sv;
                const int i0 = vb + fft_swz(k0), i1 = vb + fft_swz(k0 + h), i2 = vb + fft_swz(k0 + 2 * h),
                          i3 = vb + fft_swz(k0 + 3 * h);
                const float2 wa = tw[h + pos];                     // e^{sign pi i pos / h}
                const float2 wb = tw[2 * h + pos];                 // e^{sign pi i pos / (2 h)}
                const float2 x0 = sm[i0], x1 = sm[i1], x2 = sm[i2], x3 = sm[i3];
                const float2 a1 = make_float2(x1.x * wa.x - x1.y * wa.y, x1.x * wa.y + x1.y * wa.x);
                const float2 a3 = make_float2(x3.x * wa.x - x3.y * wa.y, x3.x * wa.y + x3.y * wa.x);
                const float2 y0 = make_float2(x0.x + a1.x, x0.y + a1.y), y1 = make_float2(x0.x - a1.x, x0.y - a1.y);
                const float2 y2 = make_float2(x2.x + a3.x, x2.y + a3.y), y3 = make_float2(x2.x - a3.x, x2.y - a3.y);
                // second stage: (y0, y2) with wb, (y1, y3) with wb e^{sign pi i / 2} = wb (sign i)
                const float2 b2 = make_float2(y2.x * wb.x - y2.y * wb.y, y2.x * wb.y + y2.y * wb.x);
                const float2 wc = make_float2(-SIGN * wb.y, SIGN * wb.x);
                const float2 b3 = make_float2(y3.x * wc.x - y3.y * wc.y, y3.x * wc.y + y3.y * wc.x);
                sm[i0] = make_float2(y0.x + b2.x, y0.y + b2.y);
                sm[i2] = make_float2(y0.x - b2.x, y0.y - b2.y);
                sm[i1] = make_float2(y1.x + b3.x, y1.y + b3.y);
                sm[i3] = make_float2(y1.x - b3.x, y1.y - b3.y);
            }
            __syncthreads();
        }
        for (int t = threadIdx.x; t < nv; t += blockDim.x) {
            const int vl = columns ? (t & (V - 1)) : (t >> log2n), k = columns ? (t >> log2V) : (t & (n - 1));
            const long long v = v0 + vl;
            if (v < nvec) a[base(v) + k * kstride] = sm[vl * sv + fft_swz(k)];
        }
        __syncthreads();
    }
}

// 256-point transforms (the planes of a 128 x 128 cube) in two radix-16 passes, 256 = 16 x 16, with
// the 16-point DFTs in registers.  Point p = j + 16 m of a vector.  Pass 1, thread (vector, j):
// Z_j[k1] = sum_m x[j + 16 m] W16^(m k1), times the twiddle W256^(j k1), into shared memory; pass 2,
// thread (vector, k1): X[k1 + 16 k2] = sum_j Z_j[k1] W16^(j k2), with W_N = e^{sign 2 pi i / N}.  One
// shared-memory round trip per transform (the general kernel takes one per pair of radix-2 stages),
// in the layout [vector][k1][j] with strides 273 and 17 complex values: both passes, in either
// thread order (rows: j fastest; columns: the vector fastest), touch 16 distinct bank slots per
// half-warp.  Loads and stores to global memory stay coalesced as in the general kernel.
constexpr int kF16VS = 273, kF16RS = 17;

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In place: x[c] <- sum_a x[a] W4^(a c) over (a0, a1, a2, a3), W4 = sign i.
template <int SIGN>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
    const float2 t = make_float2(-SIGN * d13.y, SIGN * d13.x);           // W4 (x1 - x3)
    a0 = cadd(s02, s13);
    a1 = cadd(d02, t);
    a2 = csub(s02, s13);
    a3 = csub(d02, t);
}

// In place, natural order in and out: x[k] <- sum_m x[m] W16^(m k), as m = 4a + b, k = c + 4d:
// radix-4 over a for each b, the twiddles W16^(b c), radix-4 over b for each c.
template <int SIGN>
__device__ __forceinline__ void dft16(float2 (&x)[16]) {
    constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, h = 0.70710678118654752f;   // cos, sin pi/8; cos pi/4
#pragma unroll
    for (int b = 0; b < 4; ++b) dft4<SIGN>(x[b], x[4 + b], x[8 + b], x[12 + b]);   // y_b[c] sits at x[4c + b]
    // W16^e = (cos(pi e / 8), sign sin(pi e / 8)) for e = b c
    const float2 w1 = make_float2(c1, SIGN * s1), w2 = make_float2(h, SIGN * h), w3 = make_float2(s1, SIGN * c1);
    const float2 w4 = make_float2(0.f, SIGN * 1.f), w6 = make_float2(-h, SIGN * h), w9 = make_float2(-c1, -SIGN * s1);
    x[4 + 1] = cmul(x[4 + 1], w1);    // c = 1: b = 1, 2, 3 -> e = 1, 2, 3
    x[4 + 2] = cmul(x[4 + 2], w2);
    x[4 + 3] = cmul(x[4 + 3], w3);
    x[8 + 1] = cmul(x[8 + 1], w2);    // c = 2: e = 2, 4, 6
    x[8 + 2] = cmul(x[8 + 2], w4);
    x[8 + 3] = cmul(x[8 + 3], w6);
    x[12 + 1] = cmul(x[12 + 1], w3);  // c = 3: e = 3, 6, 9
    x[12 + 2] = cmul(x[12 + 2], w6);
    x[12 + 3] = cmul(x[12 + 3], w9);
#pragma unroll
    for (int c = 0; c < 4; ++c) dft4<SIGN>(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);   // X[c + 4d] at x[4c + d]
    float2 y[16];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int d = 0; d < 4; ++d) y[c + 4 * d] = x[4 * c + d];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = y[k];
}

// Pruned: only the first 16 n_in16 points of a vector are read (the rest are zero) and only the first
// 16 n_out16 outputs are written (the rest are not needed).
template <int SIGN>
__global__ void __launch_bounds__(kPrepThreads, 2) fft256_kernel(float2* a, long long nvec, long long kstride, int log2pp,
                                                               long long vstride, long long plane_stride, int n_in16,
                                                               int n_out16) {
    __shared__ float2 sm[16 * kF16VS];
    __shared__ float2 tw[256];                       // W256^e
    const bool columns = kstride != 1;
    for (int e = threadIdx.x; e < 256; e += blockDim.x) {
        float sn, cs;
        sincospif(static_cast<float>(e) / 128.0f, &sn, &cs);   // exact power-of-two divisor
        tw[e] = make_float2(cs, SIGN * sn);
    }
    const int t = threadIdx.x;                       // 256 threads: 16 vectors x 16
    const int vl = columns ? (t & 15) : (t >> 4), q = columns ? (t >> 4) : (t & 15);   // q: j in pass 1, k1 in pass 2
    const long long pp_mask = (1LL << log2pp) - 1;
    __syncthreads();
    for (long long v0 = static_cast<long long>(blockIdx.x) * 16; v0 < nvec; v0 += static_cast<long long>(gridDim.x) * 16) {
        const long long v = v0 + vl;
        const bool live = v < nvec;
        float2* base = a + (live ? (v >> log2pp) * plane_stride + (v & pp_mask) * vstride : 0);
        float2 x[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) x[m] = live && m < n_in16 ? base[(q + 16 * m) * kstride] : make_float2(0.f, 0.f);
        dft16<SIGN>(x);                              // Z_j[k1] at x[k1], j = q
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) sm[vl * kF16VS + k1 * kF16RS + q] = cmul(x[k1], tw[(q * k1) & 255]);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 16; ++j) x[j] = sm[vl * kF16VS + q * kF16RS + j];   // k1 = q
        dft16<SIGN>(x);                              // X[k1 + 16 k2] at x[k2]
        if (live)
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2)
                if (k2 < n_out16) base[(q + 16 * k2) * kstride] = x[k2];
        __syncthreads();                             // the next group's stores reuse sm
    }
}

static int ilog2(long long x) {
    int l = 0;
    while ((1LL << l) < x) ++l;
    return l;
}

// n_in / n_out (256-point path only; 0 = n): points read and outputs written per vector.
static cudaError_t fft_smem(float2* a, long long nvec, int n, long long kstride, long long per_plane,
                            long long vstride, long long plane_stride, int sign, cudaStream_t stream, int n_in = 0,
                            int n_out = 0) {
    if (n <= 1) return cudaSuccess;                // a one-point transform is the identity
    if (n == 256) {                                // two radix-16 passes in registers
        long long grid = (nvec + 15) / 16;
        if (grid > 148LL * 16) grid = 148LL * 16;
        const int log2pp = ilog2(per_plane);
        const int in16 = (n_in > 0 ? n_in : n) / 16, out16 = (n_out > 0 ? n_out : n) / 16;
        if (sign < 0)
            fft256_kernel<-1><<<static_cast<unsigned>(grid), kPrepThreads, 0, stream>>>(a, nvec, kstride, log2pp,
                                                                                      vstride, plane_stride, in16, out16);
        else
            fft256_kernel<1><<<static_cast<unsigned>(grid), kPrepThreads, 0, stream>>>(a, nvec, kstride, log2pp,
                                                                                     vstride, plane_stride, in16, out16);
        return cudaGetLastError();
    }
    const int log2n = ilog2(n), log2pp = ilog2(per_plane);
    const int V = n >= kFftSmemPoints ? 1 : (kFftSmemPoints / n < 16 ? kFftSmemPoints / n : 16);
    const int log2V = ilog2(V);
    long long grid = (nvec + V - 1) / V;
    if (grid > 148LL * 16) grid = 148LL * 16;
    const size_t bytes = fft_smem_bytes(n, V);    // data + twiddles: up to 64 KB + 16 B
    {   // the opt-in above 48 KB of dynamic shared memory, once per device (both signs)
        static std::mutex mu;
        static std::set<int> done;
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::mutex> lk(mu);
        if (!done.count(dev)) {
            const int mx = static_cast<int>(fft_smem_bytes(kFftSmemPoints, 1));
            e = cudaFuncSetAttribute(fft_smem_kernel<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(fft_smem_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
            if (e != cudaSuccess) return e;
            done.insert(dev);
        }
    }
    if (sign < 0)
        fft_smem_kernel<-1><<<static_cast<unsigned>(grid), kPrepThreads, bytes, stream>>>(
            a, nvec, log2n, kstride, log2pp, vstride, plane_stride, log2V);
    else
        fft_smem_kernel<1><<<static_cast<unsigned>(grid), kPrepThreads, bytes, stream>>>(
            a, nvec, log2n, kstride, log2pp, vstride, plane_stride, log2V);
    return cudaGetLastError();
}

// 2-D transform of B planes [n0][n1] in place in a (b: scratch of the same size).  Sides of at
// most kFftSmemPoints points take one shared-memory pass per dimension (rows, then columns read
// in place); longer sides go through the global Stockham passes and transposes.
cudaError_t fft2_planes(float2* a, float2* b, int B, int n0, int n1, int sign, cudaStream_t stream) {
    if (n0 < 1 || n1 < 1 || (n0 & (n0 - 1)) || (n1 & (n1 - 1))) return cudaErrorInvalidValue;   // powers of two only
    if (n0 <= kFftSmemPoints && n1 <= kFftSmemPoints) {
        const long long plane = static_cast<long long>(n0) * n1;
        cudaError_t e = fft_smem(a, static_cast<long long>(B) * n0, n1, 1, n0, n1, plane, sign, stream);   // rows
        if (e != cudaSuccess) return e;
        return fft_smem(a, static_cast<long long>(B) * n1, n0, n1, n1, 1, plane, sign, stream);            // columns
    }
    const float2* r = nullptr;
    cudaError_t e = launch_fft_rows(a, b, static_cast<long long>(B) * n0, n1, sign, &r, stream);
    if (e != cudaSuccess) return e;
    float2* other = r == a ? b : a;
    const dim3 blk(32, 8);
    transpose_kernel<<<dim3((n1 + 31) / 32, (n0 + 31) / 32, B), blk, 0, stream>>>(r, other, n0, n1);   // [n1][n0]
    e = launch_fft_rows(other, const_cast<float2*>(r), static_cast<long long>(B) * n1, n0, sign, &r, stream);
    if (e != cudaSuccess) return e;
    if (r == a) {   // result of the column pass sits in a: move it to b transposed back, then copy into a
        transpose_kernel<<<dim3((n0 + 31) / 32, (n1 + 31) / 32, B), blk, 0, stream>>>(a, b, n1, n0);
        return cudaMemcpyAsync(a, b, static_cast<size_t>(B) * n0 * n1 * sizeof(float2), cudaMemcpyDeviceToDevice, stream);
    }
    transpose_kernel<<<dim3((n0 + 31) / 32, (n1 + 31) / 32, B), blk, 0, stream>>>(r, a, n1, n0);
    return cudaGetLastError();
}

// 2-D transform of B planes [n0][n1] of which only rows < in0 and columns < in1 hold non-zero values,
// keeping only outputs in rows < out0 and columns < out1 (the rest of the planes are left as they
// were).  256 x 256 planes with multiples of 16: the row pass runs over rows < in0 only, reading their
// first in1 points and writing their first out1 outputs, and the column pass over columns < out1,
// reading rows < in0 and writing rows < out0.  Other sizes: the full transform.
static cudaError_t fft2_planes_pruned(float2* a, float2* b, int B, int n0, int n1, int sign, int in0, int in1,
                                      int out0, int out1, cudaStream_t stream) {
    const bool ok = n0 == 256 && n1 == 256 && in0 > 0 && in1 > 0 && out0 > 0 && out1 > 0 && in0 <= 256 && in1 <= 256 &&
                    out0 <= 256 && out1 <= 256 && (in0 & (in0 - 1)) == 0 && (out1 & (out1 - 1)) == 0 && in1 % 16 == 0 &&
                    out0 % 16 == 0;
    if (!ok) return fft2_planes(a, b, B, n0, n1, sign, stream);
    const long long plane = 256LL * 256;
    cudaError_t e = fft_smem(a, static_cast<long long>(B) * in0, 256, 1, in0, 256, plane, sign, stream, in1, out1);   // rows
    if (e != cudaSuccess) return e;
    return fft_smem(a, static_cast<long long>(B) * out1, 256, 256, out1, 1, plane, sign, stream, in0, out0);       // columns
}

cudaError_t launch_beam_planes(const double* nu, int B, int na, int ne, double d_az, double d_el, double R,
                               double t_edge_db, float2* F, float2* work, float* peak, cudaStream_t stream,
                               bool normalise) {
    const long long plane = static_cast<long long>(na) * ne;
    const unsigned bx = static_cast<unsigned>((plane + kPrepThreads - 1) / kPrepThreads < 64 ? (plane + kPrepThreads - 1) / kPrepThreads : 64);
    aperture_kernel<<<dim3(bx, B), kPrepThreads, 0, stream>>>(F, nu, na, ne, static_cast<float>(1.0 / (na * d_az)),
                                                              static_cast<float>(1.0 / (ne * d_el)), R,
                                                              static_cast<float>(t_edge_db / 20.0));
    cudaError_t e = fft2_planes(F, work, B, na, ne, -1, stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(peak, 0, static_cast<size_t>(B) * sizeof(float), stream);
    if (e != cudaSuccess) return e;
    power_max_kernel<<<dim3(bx, B), kPrepThreads, 0, stream>>>(F, plane, peak);
    if (normalise) scale_planes_kernel<<<dim3(bx, B), kPrepThreads, 0, stream>>>(F, plane, peak);
    return cudaGetLastError();
}

cudaError_t launch_convolve_source_batch(const float* I, float* P, const double* nu, int B, int f0, int n_freq,
                                         int n_az, int n_el, double el0, double d_az, double d_el, double R,
                                         double t_edge_db, float2* K, float2* S, float2* work, float* peak,
                                         cudaStream_t stream) {
    const int na = 2 * n_az, ne = 2 * n_el;
    if (na > 65535) return cudaErrorInvalidValue;   // the plane kernels put the padded azimuth rows on grid z
    // |F|^2 left unnormalised: its peak divides the product below
    cudaError_t e = launch_beam_planes(nu + f0, B, na, ne, d_az, d_el, R, t_edge_db, K, work, peak, stream, false);
    if (e != cudaSuccess) return e;
    e = fft2_planes(K, work, B, na, ne, -1, stream);                      // transform of the beam kernel
    if (e != cudaSuccess) return e;
    source_planes_kernel<<<dim3((ne + 31) / 32, (B + 31) / 32, na), dim3(32, 8), 0, stream>>>(I, S, B, f0, n_freq, n_az,
                                                                                          n_el, el0, d_el);
    e = fft2_planes_pruned(S, work, B, na, ne, -1, n_az, n_el, na, ne, stream);    // the cube fills a quarter of the plane
    if (e != cudaSuccess) return e;
    {
        const long long plane = static_cast<long long>(na) * ne;
        const unsigned bx = static_cast<unsigned>((plane + kPrepThreads - 1) / kPrepThreads < 64 ? (plane + kPrepThreads - 1) / kPrepThreads : 64);
        multiply_scaled_kernel<<<dim3(bx, B), kPrepThreads, 0, stream>>>(S, K, plane, peak);
    }
    e = fft2_planes_pruned(S, work, B, na, ne, +1, na, ne, n_az, n_el, stream);   // only the cube's cells are gathered
    if (e != cudaSuccess) return e;
    const double A_p = 3.141592653589793 * R * R;
    const float scale = static_cast<float>(A_p * d_az * d_el / (static_cast<double>(na) * ne));   // with 1/(na ne)
    gather_planes_kernel<<<dim3((n_el + 31) / 32, (B + 31) / 32, n_az), dim3(32, 8), 0, stream>>>(S, P, B, f0, n_freq,
                                                                                                n_az, n_el, scale);
    return cudaGetLastError();
}

cudaError_t launch_smooth_screen(const float* screen, float* out, int nx, int ny, double pitch, double R,
                                 double t_edge_db, float2* K, float2* S, float2* work, double* sum,
                                 cudaStream_t stream) {
    const long long n = static_cast<long long>(nx) * ny;
    cudaError_t e = cudaMemsetAsync(sum, 0, sizeof(double), stream);
    if (e != cudaSuccess) return e;
    footprint_kernel<<<grid_for(n), kPrepThreads, 0, stream>>>(K, nx, ny, pitch, R, t_edge_db, sum);
    to_complex_kernel<<<grid_for(n), kPrepThreads, 0, stream>>>(screen, S, n);
    e = fft2_planes(K, work, 1, ny, nx, -1, stream);
    if (e != cudaSuccess) return e;
    e = fft2_planes(S, work, 1, ny, nx, -1, stream);
    if (e != cudaSuccess) return e;
    multiply_kernel<<<grid_for(n), kPrepThreads, 0, stream>>>(S, K, n);
    e = fft2_planes(S, work, 1, ny, nx, +1, stream);
    if (e != cudaSuccess) return e;
    // inverse transform is unscaled (1 / n) and the footprint unnormalised (1 / sum)
    real_part_kernel<<<grid_for(n), kPrepThreads, 0, stream>>>(S, out, n, 1.0 / static_cast<double>(n), sum);
    return cudaGetLastError();
}

}  // namespace gateau
