// Pink detector noise (Sect. 2.6, Eq. 20) as a pole-zero filter in parallel form,
//   y_n = d z_n + sum_j r_j s_j,n,   s_j,n = a_j s_j,n-1 + z_n,
// for every sequence (spaxel i, channel ch), added into out[n][i][ch].
//
// The recurrence is linear, so a run of nt samples is cut into C chunks of L
// samples scanned in parallel:
//   phase 1: each (chunk, sequence) computes its end state from a zero start;
//   phase 2: each (sequence, pole) combines the chunk states along time,
//            s_in[c+1] = a^len(c) s_in[c] + agg[c], seeded by the carried state, as a
//            warp-shuffle associative scan of the chunks' affine maps (FP32);
//   phase 3: each (chunk, sequence) reruns its chunk from s_in[c] and adds y.
// Threads of a warp own consecutive channels of one spaxel, so every sample
// step reads and writes 128 contiguous bytes of out.  The poles are held in
// pairs and updated with packed FP32 FMAs (two poles per instruction, each lane
// rounded exactly like fmaf), which halves the issue slots of the recurrence.
#include <math.h>

#include "device_common.cuh"

namespace gateau {

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Pole pair h of channel ch: (x[2h], x[2h + 1]), zero past the last pole.
__device__ __forceinline__ float2 pole_pair(const float* x, int ch, int np, int h) {
    const int j = 2 * h;
    return make_float2(j < np ? x[ch * np + j] : 0.f, j + 1 < np ? x[ch * np + j + 1] : 0.f);
}

// Samples are visited in groups of the 4 that one Philox call serves (m = n >> 2).
template <int NP>
__global__ __launch_bounds__(256, 3) void pink_phase1_kernel(DevTables T, PinkWork W, long long t0,
                                                          long long nt) {
    const long long S = static_cast<long long>(T.n_pix) * T.n_ch;
    const int np = T.n_pole;
    for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < W.C * S;
         idx += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(idx / S);
        const long long s = idx - c * S;
        const int i = static_cast<int>(s / T.n_ch), ch = static_cast<int>(s - static_cast<long long>(i) * T.n_ch);
        const long long a0 = t0 + c * W.L;
        const long long b0 = min(a0 + W.L, t0 + nt);
        constexpr int NH = NP / 2;
        float2 av[NH], st[NH];
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            av[h] = pole_pair(T.pink_a, ch, np, h);
            st[h] = make_float2(0.f, 0.f);
        }
        long long n = a0;
        // whole groups of 4 (the usual case: chunk starts are multiples of 4 when t0 is)
        if ((n & 3) == 0) {
            for (; n + 4 <= b0; n += 4) {
                const float4 z4 = pink_normals4(n >> 2, i, ch, T.key0, T.key1);
                const float zq[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 zz = make_float2(zq[q], zq[q]);
#pragma unroll
                    for (int h = 0; h < NH; ++h) st[h] = fma2(av[h], st[h], zz);
                }
            }
        }
        while (n < b0) {                             // partial groups at either end
            const long long m = n >> 2;
            const int q0 = static_cast<int>(n & 3);
            const int q1 = static_cast<int>(min(b0 - (m << 2), 4LL));
            const float4 z4 = pink_normals4(m, i, ch, T.key0, T.key1);
            for (int q = q0; q < q1; ++q) {
                const float z = f4_get(z4, q);
                const float2 zz = make_float2(z, z);
#pragma unroll
                for (int h = 0; h < NH; ++h) st[h] = fma2(av[h], st[h], zz);
            }
            n = (m << 2) + q1;
        }
        float* ag = W.agg + (c * S + s) * np;
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            if (2 * h < np) ag[2 * h] = st[h].x;
            if (2 * h + 1 < np) ag[2 * h + 1] = st[h].y;
        }
    }
}

// Phase 2: chunk c of a (sequence, pole) maps its incoming state s to a^len(c) s + agg[c], so the
// chunk states follow from composing these affine maps along time -- an associative scan, done
// here as a warp-shuffle scan: one warp per (sequence, pole), lanes = 32 consecutive chunks,
// log2(32) compose steps (f_hi o f_lo = (a_hi a_lo, a_hi b_lo + b_hi)), the running state carried
// from one block of 32 chunks to the next.  FP32: a^len = 2^(len log2 a) to ~1e-6 relative.
__global__ void pink_phase2_kernel(DevTables T, float* state, PinkWork W, long long nt) {
    const long long S = static_cast<long long>(T.n_pix) * T.n_ch;
    const int np = T.n_pole;
    const int lane = threadIdx.x & 31;
    const long long warp0 = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
    const long long n_warps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
    for (long long idx = warp0; idx < S * np; idx += n_warps) {          // warp-uniform
        const long long s = idx / np;
        const int j = static_cast<int>(idx - s * np);
        const int ch = static_cast<int>(s % T.n_ch);
        const float la = log2f(T.pink_a[ch * np + j]);                  // poles 0 < a < 1
        float carry = state[idx];
        for (int c0 = 0; c0 < W.C; c0 += 32) {
            const int c = c0 + lane;
            const bool live = c < W.C;
            float* slot = W.agg + (static_cast<long long>(live ? c : 0) * S + s) * np + j;
            // this lane's chunk map; lanes past the last chunk carry the identity
            float A = 1.f, B = 0.f;
            if (live) {
                A = exp2f(static_cast<float>(min(W.L, nt - static_cast<long long>(c) * W.L)) * la);
                B = *slot;
            }
            // inclusive scan: lane c ends with the composition of chunks c0 .. c
            for (int d = 1; d < 32; d <<= 1) {
                const float Ap = __shfl_up_sync(0xffffffffu, A, d);
                const float Bp = __shfl_up_sync(0xffffffffu, B, d);
                if (lane >= d) {
                    B = fmaf(A, Bp, B);
                    A *= Ap;
                }
            }
            // chunk c's incoming state: the composition of chunks c0 .. c - 1 applied to the carry
            float Ain = __shfl_up_sync(0xffffffffu, A, 1), Bin = __shfl_up_sync(0xffffffffu, B, 1);
            if (lane == 0) {
                Ain = 1.f;
                Bin = 0.f;
            }
            if (live) *slot = fmaf(Ain, carry, Bin);
            carry = fmaf(__shfl_sync(0xffffffffu, A, 31), carry, __shfl_sync(0xffffffffu, B, 31));
        }
        if (lane == 0) state[idx] = carry;
    }
}

// Phase 3 reads, updates and writes out one group of up to 4 samples at a time,
// with the next group's loads issued before the current group's recurrence.
constexpr int kPinkPrefetch = 128;   // samples; ~40 MB of lines in flight over the GPU, inside L2
template <int NP>
__global__ __launch_bounds__(256, 2) void pink_phase3_kernel(DevTables T, PinkWork W, long long t0,
                                                          long long nt, float* __restrict__ out) {
    const long long S = static_cast<long long>(T.n_pix) * T.n_ch;
    const int np = T.n_pole;
    const long long stride = static_cast<long long>(T.n_pix) * T.n_ch;
    for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < W.C * S;
         idx += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(idx / S);
        const long long s = idx - c * S;
        const int i = static_cast<int>(s / T.n_ch), ch = static_cast<int>(s - static_cast<long long>(i) * T.n_ch);
        const long long a0 = t0 + c * W.L;
        const long long b0 = min(a0 + W.L, t0 + nt);
        const float* ag = W.agg + (c * S + s) * np;
        constexpr int NH = NP / 2;
        float2 av[NH], rv[NH], st[NH];
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            av[h] = pole_pair(T.pink_a, ch, np, h);
            rv[h] = pole_pair(T.pink_r, ch, np, h);
            st[h] = make_float2(2 * h < np ? ag[2 * h] : 0.f, 2 * h + 1 < np ? ag[2 * h + 1] : 0.f);
        }
        const float d = T.pink_d[ch];
        float* o = out + ((a0 - t0) * T.n_pix + i) * static_cast<long long>(T.n_ch) + ch;
        long long n = a0;
        // whole groups of 4 (the usual case: chunk starts are multiples of 4 when t0 is), with the
        // next group's outputs loaded before the current group's recurrence
        if ((n & 3) == 0 && n + 4 <= b0) {
            float cur4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) cur4[q] = o[q * stride];
            while (n + 4 <= b0) {
                const bool full_next = n + 8 <= b0;
                float nxt4[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) nxt4[q] = full_next ? o[(4 + q) * stride] : 0.f;
                // and the outputs kPinkPrefetch samples ahead prefetched into L2 (the loads above
                // then wait on L2, not HBM); only within the chunk
                if (n + kPinkPrefetch + 4 <= b0) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(o + (kPinkPrefetch + q) * stride));
                }
                const float4 z4 = pink_normals4(n >> 2, i, ch, T.key0, T.key1);
                const float zq[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float z = zq[q];
                    const float2 zz = make_float2(z, z);
                    float2 ya = make_float2(d * z, 0.f), yb = make_float2(0.f, 0.f);   // two short sum chains
#pragma unroll
                    for (int h = 0; h < NH; ++h) {
                        st[h] = fma2(av[h], st[h], zz);
                        if (h & 1) yb = fma2(rv[h], st[h], yb);
                        else ya = fma2(rv[h], st[h], ya);
                    }
                    const float y = (ya.x + ya.y) + (yb.x + yb.y);
                    o[q * stride] = cur4[q] + y;
                }
                n += 4;
                o += 4 * stride;
#pragma unroll
                for (int q = 0; q < 4; ++q) cur4[q] = nxt4[q];
            }
        }
        // partial groups at either end: current group [n, n + cnt) and its loaded outputs
        int q0 = static_cast<int>(n & 3);
        int q1 = static_cast<int>(min(b0 - ((n >> 2) << 2), 4LL));
        float cur[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) cur[q] = (q >= q0 && q < q1) ? o[(q - q0) * stride] : 0.f;
        while (n < b0) {
            const long long m = n >> 2;
            const int cnt = q1 - q0;
            float* on = o + cnt * stride;
            const long long nn = (m << 2) + q1;          // first sample of the next group
            const int r1 = static_cast<int>(min(b0 - nn, 4LL));
            float nxt[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) nxt[q] = (q < r1) ? on[q * stride] : 0.f;
            const float4 z4 = pink_normals4(m, i, ch, T.key0, T.key1);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (q >= q0 && q < q1) {
                    const float z = f4_get(z4, q);
                    const float2 zz = make_float2(z, z);
                    float2 ya = make_float2(d * z, 0.f), yb = make_float2(0.f, 0.f);   // two short sum chains
#pragma unroll
                    for (int h = 0; h < NH; ++h) {
                        st[h] = fma2(av[h], st[h], zz);
                        if (h & 1) yb = fma2(rv[h], st[h], yb);
                        else ya = fma2(rv[h], st[h], ya);
                    }
                    const float y = (ya.x + ya.y) + (yb.x + yb.y);
                    o[(q - q0) * stride] = cur[q] + y;
                }
            }
            n = nn;
            o = on;
            q0 = 0;
            q1 = r1 > 0 ? r1 : 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) cur[q] = nxt[q];
        }
    }
}

// Chunking.  Every (chunk, sequence) is one thread of phases 1 and 3 doing L samples, so a phase
// runs in rounds of the threads resident on the GPU (148 SMs x the blocks per SM that the launch
// bounds pin: 3 of 256 threads for phase 1, 2 for phase 3), each round as long as one chunk.  C is
// chosen to minimise (L + 16) x (rounds of phase 3 + 0.75 rounds of phase 1) (0.75: a phase-1
// round's time against a phase-3 round's, measured; 16: a thread's fixed work -- poles, state --
// in samples), i.e. to fill the last round of both phases: with 25 x 347 sequences, 18 chunks (a
// fixed 148 K-thread target) left phase 3 three rounds with 18 of 296 blocks in the last; 26
// chunks fill three rounds of phase 3 and two of phase 1 to 99 %.  At least 64 samples per chunk;
// on a tie the fewer chunks (less state).
constexpr int kPink1Blocks = 3, kPink3Blocks = 2;
void pink_choose_chunks(long long nt, long long S, int& C, long long& L) {
    const long long cap1 = 148LL * kPink1Blocks * 256, cap3 = 148LL * kPink3Blocks * 256;
    const long long cmax = (nt + 63) / 64 > 1 ? (nt + 63) / 64 : 1;
    long long best_c = 1;
    double best = -1.0;
    for (long long c = 1; c <= cmax; ++c) {
        const long long l = ((nt + c - 1) / c + 3) / 4 * 4;
        const long long cc = (nt + l - 1) / l, U = cc * S;
        const double cost = static_cast<double>(l + 16) * (static_cast<double>((U + cap3 - 1) / cap3) +
                                                      0.75 * static_cast<double>((U + cap1 - 1) / cap1));
        if (best < 0.0 || cost < best) {
            best = cost;
            best_c = c;
        }
        if (c * S > 16 * cap3) break;                 // past 16 rounds the last one costs under 7 %
    }
    L = ((nt + best_c - 1) / best_c + 3) / 4 * 4;
    C = static_cast<int>((nt + L - 1) / L);
}

// Phases 1 and 2 (the chunk scan, which reads nothing of out) and phase 3 (the pass over out).
// (Running the scan on a second stream beside the row setup measured 0.8 ms slower per step.)
template <int NP>
static cudaError_t launch_pink_scan_np(const DevTables& T, float* state, const PinkWork& W, long long t0,
                                       long long nt, cudaStream_t stream) {
    const long long S = static_cast<long long>(T.n_pix) * T.n_ch;
    const int block = 256;
    long long grid = (W.C * S + block - 1) / block;
    if (grid > 148LL * 32) grid = 148LL * 32;
    pink_phase1_kernel<NP><<<static_cast<unsigned>(grid), block, 0, stream>>>(T, W, t0, nt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long g2 = (S * T.n_pole * 32 + block - 1) / block;      // one warp per (sequence, pole)
    if (g2 > 148LL * 32) g2 = 148LL * 32;
    pink_phase2_kernel<<<static_cast<unsigned>(g2), block, 0, stream>>>(T, state, W, nt);
    return cudaGetLastError();
}

template <int NP>
static cudaError_t launch_pink_apply_np(const DevTables& T, const PinkWork& W, long long t0, long long nt,
                                        float* out, cudaStream_t stream) {
    const long long S = static_cast<long long>(T.n_pix) * T.n_ch;
    const int block = 256;
    long long grid = (W.C * S + block - 1) / block;
    if (grid > 148LL * 32) grid = 148LL * 32;
    pink_phase3_kernel<NP><<<static_cast<unsigned>(grid), block, 0, stream>>>(T, W, t0, nt, out);
    return cudaGetLastError();
}

static cudaError_t launch_pink_scan(const DevTables& T, float* state, const PinkWork& W, long long t0,
                                    long long nt, cudaStream_t stream) {
    if (T.n_pole <= 8) return launch_pink_scan_np<8>(T, state, W, t0, nt, stream);
    if (T.n_pole <= 16) return launch_pink_scan_np<16>(T, state, W, t0, nt, stream);
    return launch_pink_scan_np<kMaxPoles>(T, state, W, t0, nt, stream);
}

static cudaError_t launch_pink_apply(const DevTables& T, const PinkWork& W, long long t0, long long nt,
                                     float* out, cudaStream_t stream) {
    if (T.n_pole <= 8) return launch_pink_apply_np<8>(T, W, t0, nt, out, stream);
    if (T.n_pole <= 16) return launch_pink_apply_np<16>(T, W, t0, nt, out, stream);
    return launch_pink_apply_np<kMaxPoles>(T, W, t0, nt, out, stream);
}

cudaError_t launch_pink(const DevTables& T, float* state, const PinkWork& W, long long t0, long long nt,
                        float* out, cudaStream_t stream) {
    const cudaError_t e = launch_pink_scan(T, state, W, t0, nt, stream);
    return e != cudaSuccess ? e : launch_pink_apply(T, W, t0, nt, out, stream);
}

}  // namespace gateau
