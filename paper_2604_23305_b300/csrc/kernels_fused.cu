// Fused split-BF16 tcgen05 kernel: steps (b)-(f) of the hot path in one pass.
//
// For a tile of 128 consecutive time samples of one spaxel and a group of NH
// channels, the kernel builds the post-cascade spectrum X[row][nu] (Sect. 2.5,
// via the exact collapse c0 + c1 (1 - eta_atm) + c2 eta_atm P_src) slice by
// slice in shared memory -- it never reaches HBM -- and contracts it on the
// 5th-generation tensor cores against the filter matrices (Sect. 2.5, Eq. 16;
// Sect. 2.6, Eq. 17):
//
//   S[row][ch] = X_hi H_hi + X_lo H_hi + X_hi H_lo         (split BF16, FP32 accumulate)
//   N[row][ch] = X_hi G + bf16(X^2) Q                       (noise terms, 1 product each)
//
// with X = X_hi + X_lo and H = H_hi + H_lo the BF16 hi/lo splits.  The
// epilogue turns S into P_KID (Eq. 16) and N into sigma (Eqs. 17-18), draws the
// white noise (Eq. 19) from Philox and writes out[n][i][ch].
//
// Warp roles (320 threads, one CTA per SM, persistent over work items):
//   warp 0      : bulk-copy producer of the pre-tiled filter operands (TMA engine)
//   warp 1      : TMEM allocator + single-thread tcgen05.mma issuer
//   warps 2..5  : spectrum producers, one thread per tile row
//   warps 6..9  : epilogue, one thread per TMEM lane (= tile row)
// Every wait is bounded: on time-out the kernel records GATEAU_STATUS_WAIT_TIMEOUT,
// stops all roles, waits (bounded) for its own copies and MMAs, frees TMEM and returns.
#include <cuda_bf16.h>
#include <math.h>

#include "device_common.cuh"

namespace gateau {

constexpr int kTileM = 128;          // rows per tile (TMEM lanes)
constexpr int kKStage = 32;          // spectral points per pipeline stage
constexpr int kAMats = 3;            // X_hi, X_lo, bf16(X^2)
constexpr int kBMats = 4;            // H_hi, H_lo, G, Q
constexpr int kThreads = 320;
constexpr int kMaxSmem = 227 * 1024;
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz

int fused_kstage() { return kKStage; }

// ---- operand layout ---------------------------------------------------------
// One (matrix, stage) block holds R rows x 32 spectral points of bf16 in
// "core matrices" of 8 rows x 16 bytes (8 points), ordered
//   [k16 step (2)][row group (R/8)][8-point chunk within the step (2)][8 rows][8 points]
// so element (r, k) sits at byte
//   (k/16)*(R/8)*256 + (r/8)*256 + ((k%16)/8)*128 + (r%8)*16 + (k%8)*2.
// For one K=16 MMA the core matrices adjacent along K are 128 B apart (leading
// byte offset) and those adjacent along rows 256 B apart (stride byte offset).
__host__ __device__ constexpr size_t core_offset(int r, int k, int R) {
    return static_cast<size_t>(k / 16) * (R / 8) * 256 + static_cast<size_t>(r / 8) * 256 +
           ((k % 16) / 8) * 128 + (r % 8) * 16 + (k % 8) * 2;
}

uint16_t f32_to_bf16_rn(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return static_cast<uint16_t>((u >> 16) | ((u & 0xffff) ? 0x40 : 0));
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return static_cast<uint16_t>(u >> 16);
}

float bf16_to_f32(uint16_t h) {
    const uint32_t u = static_cast<uint32_t>(h) << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// Host: lay out H_hi, H_lo, G, Q (FP64 [n_ch][Kp]) as [group][kstage][matrix][block].
void fused_tile_operands(const double* H, const double* G, const double* Q, int n_ch, int Kp, int n_half,
                         int n_groups, std::vector<uint16_t>& out, size_t& stage_elems) {
    const int n_ks = Kp / kKStage;
    const size_t mat_elems = static_cast<size_t>(n_half) * kKStage;
    stage_elems = mat_elems * kBMats;
    out.assign(stage_elems * n_ks * n_groups, 0);
    for (int g = 0; g < n_groups; ++g)
        for (int ks = 0; ks < n_ks; ++ks) {
            uint16_t* blk = out.data() + (static_cast<size_t>(g) * n_ks + ks) * stage_elems;
            for (int r = 0; r < n_half; ++r) {
                const int ch = g * n_half + r;
                if (ch >= n_ch) continue;
                for (int kk = 0; kk < kKStage; ++kk) {
                    const size_t src = static_cast<size_t>(ch) * Kp + ks * kKStage + kk;
                    const size_t off = core_offset(r, kk, n_half) / 2;
                    const uint16_t hhi = f32_to_bf16_rn(static_cast<float>(H[src]));
                    const double res = H[src] - static_cast<double>(bf16_to_f32(hhi));
                    blk[0 * mat_elems + off] = hhi;
                    blk[1 * mat_elems + off] = f32_to_bf16_rn(static_cast<float>(res));
                    blk[2 * mat_elems + off] = f32_to_bf16_rn(static_cast<float>(G[src]));
                    blk[3 * mat_elems + off] = f32_to_bf16_rn(static_cast<float>(Q[src]));
                }
            }
        }
}

// ---- shared-memory plan -------------------------------------------------------
struct SmemPlan {
    int n_stages;
    size_t a_bytes, b_bytes, stage_bytes, bar_off, total;
};

__host__ __device__ inline SmemPlan smem_plan(int n_half) {
    SmemPlan p;
    p.a_bytes = static_cast<size_t>(kAMats) * kTileM * kKStage * 2;
    p.b_bytes = static_cast<size_t>(kBMats) * n_half * kKStage * 2;
    p.stage_bytes = p.a_bytes + p.b_bytes;
    const size_t bar_reserve = 256;
    int ns = static_cast<int>((kMaxSmem - 1024 - bar_reserve) / p.stage_bytes);
    if (ns > 4) ns = 4;
    p.n_stages = ns;
    p.bar_off = p.stage_bytes * ns;
    p.total = p.bar_off + bar_reserve + 1024;   // + alignment slack
    return p;
}

size_t fused_smem_bytes() { return smem_plan(176).total; }

// ---- PTX wrappers ------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: returns false (and raises the abort flag) when the budget runs out
// or another role has already aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned int* status) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t_start = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t_start > kWaitCycles) {
            *abort_flag = 1;
            atomicOr(status, GATEAU_STATUS_WAIT_TIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, M=128, N from idesc, K=16, bf16 in, f32 accumulate.
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Shared-memory matrix descriptor, no swizzle (K-major core matrices).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((addr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;                    // descriptor version for tcgen05
    return d;                           // base offset 0, swizzle mode 0 (none)
}

// Instruction descriptor: kind::f16, A = B = bf16, D = f32, both K-major, M = 128.
__host__ __device__ constexpr uint32_t make_idesc(int n) {
    return (1u << 4)                                  // D format f32
           | (1u << 7)                                // A format bf16
           | (1u << 10)                               // B format bf16
           | (static_cast<uint32_t>(n >> 3) << 17)    // N / 8
           | (static_cast<uint32_t>(kTileM >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float lo_elem, float hi_elem) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// ---- work decomposition ------------------------------------------------------
struct Work {
    long long tiles_per_pix, n_items;
};

__device__ __forceinline__ void item_coords(const Work& w, int n_groups, long long it, int& pix,
                                            long long& row0, int& nrows, int& grp, long long nt) {
    const long long tile = it / n_groups;
    grp = static_cast<int>(it - tile * n_groups);
    pix = static_cast<int>(tile / w.tiles_per_pix);
    const long long tl = tile - static_cast<long long>(pix) * w.tiles_per_pix;
    row0 = tl * kTileM;                                // sample offset within the run
    const long long rem = nt - row0;
    nrows = rem < kTileM ? static_cast<int>(rem) : kTileM;
}

__global__ void __launch_bounds__(kThreads, 1)
    fused_bf16x3_kernel(DevTables T, FusedOperands F, const RowParams* __restrict__ rows, long long t0,
                        long long nt, Work work, float* __restrict__ out) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int NH = F.n_half;
    const SmemPlan sp = smem_plan(NH);
    const int NS = sp.n_stages;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + sp.bar_off);
    // barrier slots: full_a[NS], full_b[NS], empty[NS], acc_full, acc_empty
    const uint32_t bar_base = smem_u32(bars);
    auto full_a = [&](int s) { return bar_base + 8u * s; };
    auto full_b = [&](int s) { return bar_base + 8u * (NS + s); };
    auto empty_bar = [&](int s) { return bar_base + 8u * (2 * NS + s); };
    const uint32_t acc_full = bar_base + 8u * (3 * NS);
    const uint32_t acc_empty = bar_base + 8u * (3 * NS + 1);
    const uint32_t drain_bar = bar_base + 8u * (3 * NS + 2);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + sp.bar_off + 8 * (3 * NS + 3));
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + sp.bar_off + 8 * (3 * NS + 3) + 8);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full_a(s), 128);
            mbar_init(full_b(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, 128);
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const uint32_t d_sig = tmem_base;            // columns [0, NH)
    const uint32_t d_noi = tmem_base + 256;      // columns [256, 256 + NH)

    const int n_ks = T.Kp / kKStage;
    const long long my_items = work.n_items > blockIdx.x
                                   ? (work.n_items - blockIdx.x + gridDim.x - 1) / gridDim.x
                                   : 0;

    if (warp == 0) {
        // ---------------- filter-operand producer (bulk copies) ----------------
        if (lane == 0) {
            long long g = 0;     // global stage counter
            const uint32_t bytes = static_cast<uint32_t>(sp.b_bytes);
            for (long long j = 0; j < my_items && !*abort_flag; ++j) {
                const long long it = blockIdx.x + j * gridDim.x;
                const int grp = static_cast<int>(it % F.n_groups);
                const uint16_t* src = F.B + static_cast<size_t>(grp) * n_ks * F.stage_elems;
                for (int ks = 0; ks < n_ks; ++ks, ++g) {
                    const int s = static_cast<int>(g % NS);
                    const long long u = g / NS;
                    if (u > 0 && !mbar_wait(empty_bar(s), static_cast<uint32_t>((u - 1) & 1), abort_flag, T.status))
                        break;
                    mbar_arrive_expect_tx(full_b(s), bytes);
                    bulk_g2s(smem_u32(smem + s * sp.stage_bytes + sp.a_bytes), src + ks * F.stage_elems, bytes,
                             full_b(s));
                }
            }
            // Drain: every copy issued lands on its full_b barrier; wait for the
            // last NS of them (bounded) so no copy is in flight at exit.
            const long long issued = g;
            for (long long q = (issued > NS ? issued - NS : 0); q < issued; ++q) {
                const int s = static_cast<int>(q % NS);
                const uint32_t par = static_cast<uint32_t>((q / NS) & 1);
                const long long t_start = clock64();
                while (!mbar_try_wait(full_b(s), par) && clock64() - t_start < kWaitCycles) {
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = make_idesc(NH);
            long long g = 0;
            bool ok = true;
            for (long long j = 0; j < my_items && ok; ++j) {
                if (j > 0) {
                    ok = mbar_wait(acc_empty, static_cast<uint32_t>((j - 1) & 1), abort_flag, T.status);
                    if (!ok) break;
                    tc_fence_after();
                }
                for (int ks = 0; ks < n_ks; ++ks, ++g) {
                    const int s = static_cast<int>(g % NS);
                    const uint32_t par = static_cast<uint32_t>((g / NS) & 1);
                    if (!mbar_wait(full_b(s), par, abort_flag, T.status) ||
                        !mbar_wait(full_a(s), par, abort_flag, T.status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(smem + s * sp.stage_bytes);
                    const uint32_t b0 = a0 + static_cast<uint32_t>(sp.a_bytes);
                    const uint32_t a_mat = kTileM * kKStage * 2;            // bytes per A matrix
                    const uint32_t b_mat = static_cast<uint32_t>(NH) * kKStage * 2;
#pragma unroll
                    for (int kk = 0; kk < kKStage / 16; ++kk) {
                        const uint32_t a_k = kk * (kTileM / 8) * 256;
                        const uint32_t b_k = kk * (NH / 8) * 256;
                        const uint64_t xhi = smem_desc(a0 + 0 * a_mat + a_k, 128, 256);
                        const uint64_t xlo = smem_desc(a0 + 1 * a_mat + a_k, 128, 256);
                        const uint64_t xsq = smem_desc(a0 + 2 * a_mat + a_k, 128, 256);
                        const uint64_t hhi = smem_desc(b0 + 0 * b_mat + b_k, 128, 256);
                        const uint64_t hlo = smem_desc(b0 + 1 * b_mat + b_k, 128, 256);
                        const uint64_t gmat = smem_desc(b0 + 2 * b_mat + b_k, 128, 256);
                        const uint64_t qmat = smem_desc(b0 + 3 * b_mat + b_k, 128, 256);
                        const uint32_t acc = (ks > 0 || kk > 0) ? 1u : 0u;
                        tc_mma(d_sig, xhi, hhi, idesc, acc);
                        tc_mma(d_sig, xlo, hhi, idesc, 1u);
                        tc_mma(d_sig, xhi, hlo, idesc, 1u);
                        tc_mma(d_noi, xhi, gmat, idesc, acc);
                        tc_mma(d_noi, xsq, qmat, idesc, 1u);
                    }
                    tc_commit(empty_bar(s));          // stage s free once these MMAs finish
                }
                if (!ok) break;
                tc_commit(acc_full);                  // accumulators of item j complete
            }
            // Make sure no MMA is in flight at exit (bounded).
            tc_commit(drain_bar);
            const long long t_start = clock64();
            while (!mbar_try_wait(drain_bar, 0) && clock64() - t_start < kWaitCycles) {
            }
        }
    } else if (warp < 6) {
        // ---------------- spectrum producers: thread = tile row ----------------
        const int r = (warp - 2) * 32 + lane;
        long long g = 0;
        bool ok = true;
        for (long long j = 0; j < my_items && ok; ++j) {
            const long long it = blockIdx.x + j * gridDim.x;
            int pix, nrows, grp;
            long long row0;
            item_coords(work, F.n_groups, it, pix, row0, nrows, grp, nt);
            const bool valid = r < nrows;
            RowParams rp;
            if (valid) {
                rp = rows[static_cast<long long>(pix) * nt + row0 + r];
            } else {
                rp.csc = 1.f; rp.tau_j = 0; rp.tau_f = 0.f; rp.src_idx = -1; rp.src_fa = 0.f; rp.src_fe = 0.f;
            }
            if (rp.tau_j < 0 || rp.tau_j > T.n_pwv - 2) {
                atomicOr(T.status, GATEAU_STATUS_BAD_INDEX);
                rp.tau_j = 0;
            }
            const float* tA = T.tau + static_cast<long long>(rp.tau_j) * T.Kp;
            const float* tB = tA + T.Kp;
            const bool has_src = valid && rp.src_idx >= 0;
            const float fa = rp.src_fa, fe = rp.src_fe;
            const float w00 = (1.f - fa) * (1.f - fe), w10 = fa * (1.f - fe), w01 = (1.f - fa) * fe, w11 = fa * fe;
            const float* s00 = T.cube + (has_src ? rp.src_idx : 0);
            const float* s10 = s00 + static_cast<long long>(T.n_el) * T.Kp;
            const float* s01 = s00 + T.Kp;
            const float* s11 = s10 + T.Kp;
            const float csc = rp.csc, tf = rp.tau_f;
            for (int ks = 0; ks < n_ks; ++ks, ++g) {
                const int s = static_cast<int>(g % NS);
                const long long u = g / NS;
                if (u > 0 && !mbar_wait(empty_bar(s), static_cast<uint32_t>((u - 1) & 1), abort_flag, T.status)) {
                    ok = false;
                    break;
                }
                uint8_t* a0 = smem + s * sp.stage_bytes;
#pragma unroll
                for (int kc = 0; kc < kKStage / 8; ++kc) {
                    const int k = ks * kKStage + kc * 8;
                    float x[8];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int kq = k + 4 * h;
                        const float4 ta = *reinterpret_cast<const float4*>(tA + kq);
                        const float4 tb = *reinterpret_cast<const float4*>(tB + kq);
                        const float4 c0 = __ldg(reinterpret_cast<const float4*>(T.c0 + kq));
                        const float4 c1 = __ldg(reinterpret_cast<const float4*>(T.c1 + kq));
                        const float4 c2 = __ldg(reinterpret_cast<const float4*>(T.c2 + kq));
                        float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (has_src) {
                            const float4 q00 = *reinterpret_cast<const float4*>(s00 + kq);
                            const float4 q10 = *reinterpret_cast<const float4*>(s10 + kq);
                            const float4 q01 = *reinterpret_cast<const float4*>(s01 + kq);
                            const float4 q11 = *reinterpret_cast<const float4*>(s11 + kq);
                            p.x = w00 * q00.x + w10 * q10.x + w01 * q01.x + w11 * q11.x;
                            p.y = w00 * q00.y + w10 * q10.y + w01 * q01.y + w11 * q11.y;
                            p.z = w00 * q00.z + w10 * q10.z + w01 * q01.z + w11 * q11.z;
                            p.w = w00 * q00.w + w10 * q10.w + w01 * q01.w + w11 * q11.w;
                        }
#define GATEAU_FX(i, c)                                          \
    {                                                            \
        const float tau = ta.c + tf * (tb.c - ta.c);             \
        const float e = __expf(-csc * tau);                      \
        x[4 * h + i] = c0.c + c1.c * (1.f - e) + c2.c * e * p.c; \
    }
                        GATEAU_FX(0, x) GATEAU_FX(1, y) GATEAU_FX(2, z) GATEAU_FX(3, w)
#undef GATEAU_FX
                    }
                    uint32_t hi[4], lo[4], sq[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float xa = x[2 * q], xb = x[2 * q + 1];
                        const __nv_bfloat162 h2 = __floats2bfloat162_rn(xa, xb);
                        hi[q] = *reinterpret_cast<const uint32_t*>(&h2);
                        lo[q] = pack_bf16(xa - __low2float(h2), xb - __high2float(h2));
                        sq[q] = pack_bf16(xa * xa, xb * xb);
                    }
                    const size_t off = core_offset(r, kc * 8, kTileM);
                    *reinterpret_cast<uint4*>(a0 + 0 * (kTileM * kKStage * 2) + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<uint4*>(a0 + 1 * (kTileM * kKStage * 2) + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                    *reinterpret_cast<uint4*>(a0 + 2 * (kTileM * kKStage * 2) + off) = make_uint4(sq[0], sq[1], sq[2], sq[3]);
                }
                fence_proxy_async();
                mbar_arrive(full_a(s));
            }
        }
    } else {
        // ---------------- epilogue: thread = TMEM lane = tile row ----------------
        const int quad = warp & 3;                   // TMEM lane quadrant this warp may access
        const int r = quad * 32 + lane;
        const bool white = (T.noise_flags & GATEAU_NOISE_WHITE) != 0;
        for (long long j = 0; j < my_items; ++j) {
            // tcgen05.ld is warp-collective: take the wait's outcome warp-uniformly.
            const bool ok = mbar_wait(acc_full, static_cast<uint32_t>(j & 1), abort_flag, T.status);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            const long long it = blockIdx.x + j * gridDim.x;
            int pix, nrows, grp;
            long long row0;
            item_coords(work, F.n_groups, it, pix, row0, nrows, grp, nt);
            const long long n = t0 + row0 + r;
            float* orow = out + ((row0 + r) * T.n_pix + pix) * static_cast<long long>(T.n_ch);
            const int ch_base = grp * NH;
            for (int c = 0; c < NH; c += 16) {
                float sv[16], nv[16];
                const uint32_t lane_off = static_cast<uint32_t>(quad * 32) << 16;
                tmem_ld16(d_sig + lane_off + c, sv);
                tmem_ld16(d_noi + lane_off + c, nv);
                tmem_wait_ld();
                if (r < nrows) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int ch0 = ch_base + c + 4 * q;
                        if (ch0 >= T.n_ch) break;
                        float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (white) z = white_normals4(n, pix, ch0 >> 2, T.key0, T.key1);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int ch = ch0 + e;
                            if (ch < T.n_ch) {
                                const float pk = T.kb1e9 * sv[4 * q + e];
                                const float sigma = T.kB * sqrtf(T.noise_scale * fmaxf(nv[4 * q + e], 0.f));
                                orow[ch] = fmaf(sigma, f4_get(z, e), pk);
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(acc_empty);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
    }
}

cudaError_t launch_fused_bf16x3(const DevTables& T, const FusedOperands& F, const RowParams* rows, long long t0,
                                long long nt, float* out, int n_sm, cudaStream_t stream) {
    const SmemPlan sp = smem_plan(F.n_half);
    if (sp.n_stages < 2) return cudaErrorInvalidConfiguration;
    Work w;
    w.tiles_per_pix = (nt + kTileM - 1) / kTileM;
    w.n_items = w.tiles_per_pix * T.n_pix * F.n_groups;
    if (w.n_items == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fused_bf16x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sp.total));
    if (e != cudaSuccess) return e;
    long long grid = w.n_items < n_sm ? w.n_items : n_sm;
    fused_bf16x3_kernel<<<static_cast<unsigned>(grid), kThreads, sp.total, stream>>>(T, F, rows, t0, nt, w, out);
    return cudaGetLastError();
}

}  // namespace gateau
