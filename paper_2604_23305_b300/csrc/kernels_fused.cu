// Fused split-BF16 tcgen05 kernel: steps (b)-(f) of the hot path in one pass.
//
// For a tile of 128 consecutive time samples of one spaxel and a group of NH
// channels, the kernel builds the post-cascade spectrum (Sect. 2.5, via the
// exact collapse X = c0 + c1 (1 - eta_atm) + c2 eta_atm P_src) as its difference
// D = X - X_ref from the plan's source-free reference spectrum
// X_ref = c0 + c1 (1 - e_ref), i.e. D = c_ref - c1 eta_atm + eta_atm P'_src, slice
// by slice in shared memory -- it never reaches HBM -- and contracts it on the
// 5th-generation tensor cores against the filter matrices (Sect. 2.5, Eq. 16;
// Sect. 2.6, Eq. 17):
//
//   S[row][ch] = D_hi H_hi + D_lo H_hi + D_hi H_lo         (split BF16, FP32 accumulate)
//   N[row][ch] = D_hi G' + bf16(D_hi^2) Q                   (noise terms, 1 product each)
//
// with D = D_hi + D_lo and H = H_hi + H_lo the BF16 hi/lo splits and
// G' = G + 2 Q X_ref (the cross term of X^2 = (D + X_ref)^2).  D is small next to
// X wherever the sky is near its mean, so the rounding of the split products is
// relative to the sky's fluctuation, not to the whole loading, and the faint
// source term survives it.  The epilogue adds the reference's integrals
// (per-channel constants), turns S into P_KID (Eq. 16) and N into sigma
// (Eqs. 17-18), adds the white noise (Eq. 19, Philox normals drawn while the
// item's MMAs run and parked in free TMEM columns) and writes out[n][i][ch].
//
// Warp roles (512 threads, one CTA per SM, persistent over work items):
//   warp 0        : one thread issuing bulk copies of the pre-tiled filter operands (B ring)
//   warp 1        : TMEM allocator + single-thread tcgen05.mma issuer (a stage's five MMAs in one
//                   asm block; it and the warp-0 loader poll their barriers: both threads are on
//                   the kernel's critical chain)
//   warp 2        : one thread issuing tensor copies of the tile's opacity rows and cube texel
//                   box (input ring); each spinning role has a warp of its own
//   warp 3        : shared tiles only: one thread copying this CTA's finished rows of each
//                   stage into the peer CTA's shared memory
//   warps 4..11   : spectrum producers; each warp signals its own rows (no CTA-wide barrier).
//                   With 177-352 channels the two channel groups of a tile run on the two CTAs
//                   of a cluster: each CTA builds half of the tile's rows, 16 rows per warp,
//                   and warp 3 ships them into the peer's shared memory (one build per row)
//   warps 12..15  : shared tiles: a third producer group; independent CTAs: epilogue only.
//                   The epilogue of each item is shared by warps 4..15 (three per TMEM quadrant)
// The input ring runs ahead of the producers, the A/B ring behind them, so the
// producers read their gathers from shared memory.  A tile whose rows span one or two
// opacity-table rows, or stay in one row of cube cells, stages the smaller box of each
// (less for the SM to take in per stage); rows outside the staged boxes read global memory.
// Every wait is bounded: on time-out the kernel records GATEAU_STATUS_WAIT_TIMEOUT,
// stops all roles, waits (bounded) for its own copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include "device_common.cuh"

namespace gateau {

constexpr int kTileM = kTileRows;    // rows per tile (TMEM lanes)
constexpr int kKStage = 16;          // spectral points per pipeline stage (one K=16 MMA step)
constexpr int kAMats = 3;            // D_hi, D_lo, bf16(D_hi^2)
constexpr int kBMats = 4;            // H_hi, H_lo, G', Q
constexpr int kProdWarps = 8;
constexpr int kProdWarp0 = 4;               // warps 0..3: operand TMA, MMA, input TMA, peer copier
constexpr int kEpiWarp0 = kProdWarp0 + kProdWarps;
constexpr int kThreads = (kEpiWarp0 + 4) * 32;
constexpr int kMaxSmem = 218 * 1024;   // a 2-CTA cluster launch with 223 KB per CTA was refused; stay below
constexpr int kInSlots = 6;          // input-ring depth (stages of staged gathers)
// Staged rows are 20 points wide (80 B): the 16 points of the stage plus 4 that
// are never read.  With a 20-word row stride, successive texels start on
// different shared-memory banks, so lanes reading different texels at the same
// point do not conflict.
constexpr int kBoxW = 20;
constexpr int kCubeBoxBytes = kCubeBoxAz * kCubeBoxEl * kBoxW * 4;    // 3840
constexpr int kCubeBoxBytesS = kCubeBoxAz * kCubeBoxElS * kBoxW * 4;  // 1920: the small box, at the slot's start
constexpr int kTauBoxBytes = 2 * kTauBoxRows * kBoxW * 4;             // (tau_j, dtau_j) rows: 1280
constexpr int kTauBoxBytesS = 2 * kTauBoxRowsS * kBoxW * 4;           // the small box: 320
constexpr int kConstBytes = 2 * kKStage * 4;                          // c_ref and c1 of the stage
constexpr int kTauOff = kCubeBoxBytes;
constexpr int kConstOff = kCubeBoxBytes + kTauBoxBytes;
constexpr int kInSlotBytes = (kConstOff + kConstBytes + 127) / 128 * 128;
constexpr long long kWaitCycles = kDefaultWaitCycles;   // drains on the exit path: ~2 s at 2 GHz
// Grace on the exit path of an aborted shared tile: a peer's row copies into this CTA complete on
// stage barriers that an aborted loader may never have armed, so no drain reports them; each CTA
// waits this long after its last copy was issued before it arrives on the final cluster barrier,
// which the peer must pass before it can exit (a 2 KB copy lands in about a microsecond).
constexpr long long kAbortGraceCycles = 2000000LL;      // ~1 ms

int fused_kstage() { return kKStage; }

// ---- operand layout ---------------------------------------------------------
// One (matrix, stage) block holds R rows x 16 spectral points of bf16 in "core
// matrices" of 8 rows x 16 bytes (8 points), ordered
//   [row group (R/8)][8-point half of the slice (2)][8 rows][8 points]
// so element (r, k) sits at byte (r/8)*256 + (k/8)*128 + (r%8)*16 + (k%8)*2.
// For the K=16 MMA the core matrices adjacent along K are 128 B apart (leading
// byte offset) and those adjacent along rows 256 B apart (stride byte offset);
// either reading of the two offsets stays inside the block.
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

// Host: lay out H_hi, H_lo, G', Q (formed per element, FP64) as [group][kstage][matrix][block].
void fused_tile_operands(const FilterOperands& f, int n_ch, int Kp, int n_half, int n_groups,
                         std::vector<uint16_t>& out, size_t& stage_elems) {
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
                    const int k = ks * kKStage + kk;
                    if (k >= f.nf) continue;                 // zero past the grid (out is zeroed)
                    double h, g, q;
                    f.at(ch, k, h, g, q);
                    const size_t off = core_offset(r, kk, n_half) / 2;
                    const uint16_t hhi = f32_to_bf16_rn(static_cast<float>(h));
                    const double res = h - static_cast<double>(bf16_to_f32(hhi));
                    blk[0 * mat_elems + off] = hhi;
                    blk[1 * mat_elems + off] = f32_to_bf16_rn(static_cast<float>(res));
                    blk[2 * mat_elems + off] = f32_to_bf16_rn(static_cast<float>(f.gprime(g, q, k)));
                    blk[3 * mat_elems + off] = f32_to_bf16_rn(static_cast<float>(q));
                }
            }
        }
}

// Host: tensor maps of the opacity table and the cube for the staged gathers.
bool fused_encode_input_maps(const float* tau, int n_pwv, const float* cube, int n_az, int n_el, int Kp,
                             TensorMapBytes* tm_tau, TensorMapBytes* tm_tau_s, TensorMapBytes* tm_cube,
                             TensorMapBytes* tm_cube_s,
                             std::string& err) {
    static_assert(sizeof(CUtensorMap) == sizeof(TensorMapBytes), "tensor map size");
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        err = "cuTensorMapEncodeTiled unavailable";
        return false;
    }
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    Encode encode = reinterpret_cast<Encode>(fn);
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int small = 0; small < 2; ++small) {
        const cuuint64_t dims[2] = {static_cast<cuuint64_t>(Kp), static_cast<cuuint64_t>(2 * n_pwv)};
        const cuuint64_t strides[1] = {static_cast<cuuint64_t>(Kp) * 4};
        const cuuint32_t box[2] = {kBoxW, static_cast<cuuint32_t>(2 * (small ? kTauBoxRowsS : kTauBoxRows))};
        CUresult r = encode(reinterpret_cast<CUtensorMap*>(small ? tm_tau_s : tm_tau), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                            const_cast<float*>(tau), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            err = "tensor map of the opacity table: CUresult " + std::to_string(static_cast<int>(r));
            return false;
        }
    }
    for (int small = 0; small < 2; ++small) {
        const cuuint64_t dims[3] = {static_cast<cuuint64_t>(Kp), static_cast<cuuint64_t>(n_el),
                                    static_cast<cuuint64_t>(n_az)};
        const cuuint64_t strides[2] = {static_cast<cuuint64_t>(Kp) * 4, static_cast<cuuint64_t>(Kp) * 4 * n_el};
        const cuuint32_t box[3] = {kBoxW, static_cast<cuuint32_t>(small ? kCubeBoxElS : kCubeBoxEl), kCubeBoxAz};
        CUresult r = encode(reinterpret_cast<CUtensorMap*>(small ? tm_cube_s : tm_cube), CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                            3, const_cast<float*>(cube), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            err = "tensor map of the cube: CUresult " + std::to_string(static_cast<int>(r));
            return false;
        }
    }
    return true;
}

// ---- shared-memory plan -------------------------------------------------------
// The spectrum rows (A: D_hi, D_lo, bf16(D_hi^2)) and the filter operands (B: H_hi, H_lo, G', Q)
// of a stage live in two rings of their own.  A slot is reused only after the rows have been
// built again (and, for a shared tile, copied from the peer), a long round trip, so the A ring
// is the deeper one; a B slot only waits for its copy from L2.
struct SmemPlan {
    int nsa, nsb;                       // A-ring and B-ring depths (nsb <= nsa)
    size_t a_bytes, b_bytes, b_off, in_off, bar_off, total;
};

constexpr size_t kBarReserve = 512;     // mbarriers, TMEM address slot and abort flag
constexpr int kMaxHalf = 176;           // channels per group: 2 x 176 accumulator columns + parked normals
// The reference spectrum's per-channel P_KID and N of a CTA's channel group sit in a static shared
// array (1408 B, before the dynamic rings: the dynamic base is aligned up to 1024 B inside the slack
// the plan reserves) in a single-job launch of shared tiles, where a CTA's group is fixed: the epilogue
// reads them from shared memory instead of issuing global loads between its TMEM reads and its stores.
// (Global loads there cost ~0.9 ms per ifu25 launch, measured with clock64 counters.)

// Ring depths for channel groups of n_half: the deepest B ring up to ring_b (2..kMaxRingB) whose
// stages leave room for at least as many A slots (at most 8, whole pairs).
__host__ __device__ constexpr SmemPlan smem_plan(int n_half, int ring_b = kDefaultRingB) {
    SmemPlan p{};
    p.a_bytes = static_cast<size_t>(kAMats) * kTileM * kKStage * 2;
    p.b_bytes = static_cast<size_t>(kBMats) * n_half * kKStage * 2;
    const size_t bar_reserve = kBarReserve;
    const size_t in_bytes = static_cast<size_t>(kInSlots) * kInSlotBytes;
    const long long avail = static_cast<long long>(kMaxSmem) - 1024 - bar_reserve - in_bytes;
    p.nsa = 0;
    p.nsb = 0;
    for (int nsb = ring_b; nsb >= 2; --nsb) {
        long long nsa = (avail - static_cast<long long>(nsb) * p.b_bytes) / static_cast<long long>(p.a_bytes);
        if (nsa > 8) nsa = 8;
        nsa &= ~1LL;                               // whole stage pairs
        if (nsa >= nsb) {
            p.nsa = static_cast<int>(nsa);
            p.nsb = nsb;
            break;
        }
    }
    p.b_off = p.a_bytes * p.nsa;
    p.in_off = p.b_off + p.b_bytes * p.nsb;
    p.bar_off = p.in_off + in_bytes;
    p.total = p.bar_off + bar_reserve + 1024;   // + alignment slack
    return p;
}

size_t fused_smem_bytes() { return smem_plan(kMaxHalf).total; }

int fused_ring_depths(int n_half, int ring_b, int* nsa) {
    const SmemPlan p = smem_plan(n_half, ring_b);
    if (nsa) *nsa = p.nsa;
    return p.nsb;
}

// What the barrier protocol below assumes of the ring depths (each checked at compile time for
// every group width the plan can choose, and again at launch):
//  * the MMA issuer takes stage pairs: the A ring holds whole pairs (nsa even), so a pair's
//    stage-full and stage-free barriers serve slots 2p and 2p + 1;
//  * nsb <= nsa: the operand loader refills the B slot of stage g after the MMAs of stage
//    g - nsb, by which time the A-slot pair barrier of stage g has left the phase of stage
//    g - nsa, and no barrier a loader or the issuer waits on can run two phases ahead of it;
//  * an item's first nsa stages are built before the previous item's epilogue (kPre = nsa): their
//    slots are freed by the previous item's MMAs alone, which need no epilogue;
//  * the barriers (3 nsa + 2 kInSlots, three item barriers, the TMEM slot and abort flag, nsa / 2
//    first-stage B releases) fit the reserved bytes;
//  * a pair's expected transaction bytes (B operands and, for a shared tile, the peer's rows of
//    both stages) stay below the mbarrier's 2^20 limit;
//  * the rings start on 1024-byte (A) and 16-byte (B, bulk copies) boundaries.
constexpr bool ring_protocol_ok(const SmemPlan& p) {
    return p.nsa >= 2 && p.nsa % 2 == 0 && p.nsb >= 2 && p.nsb <= p.nsa &&
           8 * (3 * p.nsa + 2 * kInSlots + 5 + p.nsa / 2) <= static_cast<int>(kBarReserve) &&
           2 * (p.b_bytes + static_cast<size_t>(kAMats) * kTileM * kKStage) < (size_t(1) << 20) &&
           p.a_bytes % 1024 == 0 && p.b_off % 1024 == 0 && p.b_bytes % 16 == 0 && p.in_off % 128 == 0 &&
           p.total <= static_cast<size_t>(kMaxSmem);
}

constexpr bool ring_protocol_ok_for_all_groups() {
    for (int nh = 16; nh <= kMaxHalf; nh += 16)
        for (int rb = 2; rb <= kMaxRingB; ++rb)
            if (!ring_protocol_ok(smem_plan(nh, rb))) return false;
    return true;
}

static_assert(ring_protocol_ok_for_all_groups(), "ring depths break the barrier protocol");
static_assert(kTileM == 128, "M = 128 MMAs: one TMEM lane per tile row");
static_assert(kProdWarps == 8 && kThreads == 512, "warp roles: 4 single-thread roles, 8 producers, 4 epilogue");
static_assert(kThreads / 32 - kProdWarp0 == 4 + kProdWarps, "acc_empty counts every epilogue-sharing warp");
static_assert(3 * (kProdWarps / 2) == kThreads / 32 - kProdWarp0 && 16 * (kProdWarps / 2) == kTileM / 2,
              "shared tiles: three groups of four producer warps, 16 rows each, build a CTA's 64 rows");
static_assert(16 * kProdWarps == kTileM, "independent CTAs: eight producer warps build the 128 rows");
static_assert(kInSlotBytes % 128 == 0, "input slots start on 128-byte boundaries (tensor copies)");

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

// Bounded wait: returns false (and raises the abort flag) when the budget (clock64 cycles, a
// run-time parameter) runs out or another role has already aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned int* status, long long budget) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t_start = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t_start > budget) {
            *abort_flag = 1;
            atomicOr(status, GATEAU_STATUS_WAIT_TIMEOUT);
            return false;
        }
    }
}

// Non-blocking test of a phase (mbarrier.test_wait: the thread is never suspended).
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded polling wait for the single-thread roles on the kernel's critical chain (the MMA issuer
// waiting for stage data, the filter-operand loader waiting for a free B slot): polling with
// test_wait sees a completed phase sooner than a thread suspended in try_wait is resumed, which
// measured ~0.7 ms less per ifu25 launch.  Budget and abort as in mbar_wait.
__device__ __forceinline__ bool mbar_wait_poll(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                               unsigned int* status, long long budget) {
    if (mbar_test(bar, parity)) return true;
    const long long t_start = clock64();
    while (true) {
        for (int i = 0; i < 16; ++i)
            if (mbar_test(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t_start > budget) {
            *abort_flag = 1;
            atomicOr(status, GATEAU_STATUS_WAIT_TIMEOUT);
            return false;
        }
    }
}

// Bounded wait for a long-pending phase (the epilogue's wait for a finished item): between
// polls the thread sleeps, so idle waiters do not take shared-memory issue slots from the
// roles on the critical path.
__device__ __forceinline__ bool mbar_wait_idle(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                               unsigned int* status, long long budget) {
    const long long t_start = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t_start > budget) {
            *abort_flag = 1;
            atomicOr(status, GATEAU_STATUS_WAIT_TIMEOUT);
            return false;
        }
        __nanosleep(256);
    }
}

// Bounded wait used on the exit path (no abort check).
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
    const long long t_start = clock64();
    while (!mbar_try_wait(bar, parity) && clock64() - t_start < kWaitCycles) {
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

__device__ __forceinline__ void tensor2d_g2s(uint32_t dst, const void* tmap, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tensor3d_g2s(uint32_t dst, const void* tmap, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Peer CTA's shared::cluster address of a local shared::cta address.
__device__ __forceinline__ uint32_t mapa_peer(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release;\nbarrier.cluster.wait.acquire;" ::: "memory");
}

// Local shared memory -> peer CTA's shared memory, completing on the peer's mbarrier.
__device__ __forceinline__ void bulk_s2peer(uint32_t dst_cluster, uint32_t src_cta, uint32_t bytes,
                                            uint32_t bar_cluster) {
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst_cluster),
        "r"(src_cta), "r"(bytes), "r"(bar_cluster)
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

// Commit arriving on the barrier at the same offset in both CTAs of a 2-CTA cluster.
__device__ __forceinline__ void tc_commit_pair(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            bar),
        "h"(static_cast<uint16_t>(3))
        : "memory");
}

// One 16-point stage of the fused contraction, issued by one thread in one block: the three S
// products D_hi H_hi, D_lo H_hi, D_hi H_lo into d_sig and the two N products D_hi G', bf16(D_hi^2) Q
// into d_noi (M = 128, N and the types from idesc, K = 16).  Descriptors come as their low words
// (start address and leading byte offset; the slot offsets are added there, without carry since
// shared addresses stay below 256 KB) and the common high word (stride byte offset, version):
// the issuing thread is on the kernel's critical path, so the block keeps its work small.
// acc = 0 overwrites the accumulators (the first stage of an item); the other products accumulate.
__device__ __forceinline__ void tc_mma_stage(uint32_t d_sig, uint32_t d_noi, uint32_t xhi, uint32_t xlo,
                                             uint32_t xsq, uint32_t hhi, uint32_t hlo, uint32_t gmat,
                                             uint32_t qmat, uint32_t dhi, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p, t;\n.reg .b64 a0, a1, a2, b0, b1, b2, b3;\n"
        "setp.ne.b32 p, %11, 0;\n"
        "setp.eq.b32 t, %11, %11;\n"
        "mov.b64 a0, {%2, %9};\nmov.b64 a1, {%3, %9};\nmov.b64 a2, {%4, %9};\n"
        "mov.b64 b0, {%5, %9};\nmov.b64 b1, {%6, %9};\nmov.b64 b2, {%7, %9};\nmov.b64 b3, {%8, %9};\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], a0, b0, %10, p;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], a1, b0, %10, t;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], a0, b1, %10, t;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%1], a0, b2, %10, p;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%1], a2, b3, %10, t;\n}" ::"r"(d_sig),
        "r"(d_noi), "r"(xhi), "r"(xlo), "r"(xsq), "r"(hhi), "r"(hlo), "r"(gmat), "r"(qmat), "r"(dhi), "r"(idesc),
        "r"(acc)
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

// 16 lanes x 8 columns (the 16x256b shape): thread t gets lane base + t/4 (registers 0, 1) and
// base + t/4 + 8 (registers 2, 3), columns 2 (t % 4) + {0, 1}.
__device__ __forceinline__ void tmem_ld16x256b_x1(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.16x256b.x1.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}

// The wait for this thread's TMEM loads, naming the 12 registers they fill: the compiler sees
// them written here, so no use of them is scheduled before the data has arrived.
__device__ __forceinline__ void tmem_wait_ld_regs(uint32_t (&a)[4], uint32_t (&b)[4], uint32_t (&c)[4]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]),
                   "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
                 :
                 : "memory");
}

// The store of the same shape: register i of thread t goes to the cell that tmem_ld16x256b_x1
// reads into register i of thread t.
__device__ __forceinline__ void tmem_st16x256b_x1(uint32_t taddr, const float (&v)[4]) {
    asm volatile("tcgen05.st.sync.aligned.16x256b.x1.b32 [%0], {%1,%2,%3,%4};"
                 ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                   "r"(__float_as_uint(v[3]))
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float lo_elem, float hi_elem) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// 2^x on the special-function unit (relative error ~2^-22 over the range used here).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---- work decomposition ------------------------------------------------------
// A launch runs the work items of one or more plans' runs ("jobs"; several when a server batches
// the time chunks of its requests into one launch).  Everything an item reads of its plan lives in
// its job, in the kernel's parameter space (the tensor maps must be there or in global memory for
// the tensor copies).  Items are numbered job by job; a CTA (or a cluster, for shared tiles) takes
// every gridDim-th item of that numbering, whatever job it belongs to.
struct __align__(128) FusedJob {   // (CUtensorMap is 128-byte aligned)
    CUtensorMap tm_tau, tm_tau_s, tm_cube, tm_cube_s;   // staged inputs of this plan (full and small boxes)
    DevTables T;
    FusedOperands F;
    const RowParams* rows;
    const TileInfo* tiles;
    long long t0, nt;                  // the run: samples t0 .. t0 + nt - 1
    float* out;                        // [nt][n_pix][n_ch]
    long long tiles_per_pix;
    long long item0, n_items;          // this job's items in the launch's numbering
};

constexpr int kMaxJobs = 28;           // 28 jobs of 1152 bytes stay inside the 32 KB of kernel parameters

template <int NJ>
struct FusedLaunch {
    FusedJob job[NJ];
    int n_jobs;
    int layout_half;                   // channels per CTA that size the rings: the widest job's
    int ring_b;                        // deepest B ring the layout may take (the jobs' smallest choice)
    long long n_items;                 // items of all jobs
    long long wait_cycles;             // budget of each pipeline wait (clock64 cycles)
};
static_assert(sizeof(FusedLaunch<kMaxJobs>) <= 32764, "the job table must fit the kernel parameter space");

// Item li of job J: li = (tile-in-pixel * n_pix + pix) * n_groups + group.  A job's items are
// walked time tile by time tile, all spaxels of one time tile next to each other.  The CTAs
// resident at one moment then look at one stretch of the scan -- the IFU's spaxels see
// neighbouring cube texels -- and write neighbouring output rows ([n][pix][ch]), so cube boxes hit
// L2 and output lines fill together.  tile = pix * tiles_per_pix + tile-in-pixel indexes the
// TileInfo records.
__device__ __forceinline__ void item_coords(const FusedJob& J, long long li, long long& tile, int& pix,
                                            long long& row0, int& nrows, int& grp) {
    const int n_groups = J.F.n_groups;
    const long long u = li / n_groups;
    grp = static_cast<int>(li - u * n_groups);
    const long long tl = u / J.T.n_pix;
    pix = static_cast<int>(u - tl * J.T.n_pix);
    tile = static_cast<long long>(pix) * J.tiles_per_pix + tl;
    row0 = tl * kTileM;                                // sample offset within the run
    const long long rem = J.nt - row0;
    nrows = rem < kTileM ? static_cast<int>(rem) : kTileM;
}

template <int kShare, int NJ>
__global__ void __launch_bounds__(kThreads, 1) fused_bf16x3_kernel(const __grid_constant__ FusedLaunch<NJ> L) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const SmemPlan sp = smem_plan(L.layout_half, L.ring_b);   // ring layout: the widest job's channel group
    const int NS = sp.nsa;                       // A-ring depth
    const int NSB = sp.nsb;                      // B-ring depth
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + sp.bar_off);
    const uint32_t bar_base = smem_u32(bars);
    // One "stage full" barrier per ring slot: the operand copy's arrival (+ its bytes) and the
    // spectrum rows' arrival(s) (+ the peer's bytes for a shared tile), so the MMA issuer waits once.
    // The MMA issuer takes two 16-point stages per handshake (10 MMAs per wait and commit):
    // the stage-full and stage-free barriers belong to pairs of A slots (2p, 2p + 1).
    auto full_a = [&](int s) { return bar_base + 8u * (s >> 1); };                 // per A-slot pair
    auto empty_bar = [&](int s) { return bar_base + 8u * (NS + (s >> 1)); };       // per A-slot pair
    auto full_in = [&](int s) { return bar_base + 8u * (2 * NS + s); };
    auto empty_in = [&](int s) { return bar_base + 8u * (2 * NS + kInSlots + s); };
    auto rows_ready = [&](int s) { return bar_base + 8u * (2 * NS + 2 * kInSlots + s); };   // per A slot
    const int nb = 3 * NS + 2 * kInSlots;
    const uint32_t acc_full = bar_base + 8u * nb;
    const uint32_t acc_empty = bar_base + 8u * (nb + 1);
    const uint32_t drain_bar = bar_base + 8u * (nb + 2);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + sp.bar_off + 8 * (nb + 3));
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + sp.bar_off + 8 * (nb + 3) + 8);
    // B slot of the first stage of a pair: free once that stage's MMAs are done, which a local
    // commit between the pair's two stages reports half a pair before the pair's stage-free
    // barrier (B streaming is latency-bound, so the earlier refill shortens every stage).  The
    // same early release of the first A slot (a multicast commit) measured slower.
    auto bfree_first = [&](int s) { return bar_base + 8u * (nb + 5 + (s >> 1)); };   // per A-slot pair

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int share = kShare;
    const uint32_t rank = share ? cluster_rank() : 0u;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; s += 2) {
            // per stage of the pair: the operand copy's arrival (its bytes and, for a shared tile,
            // the peer's rows) + one per producer warp (independent CTA) or the copier's (shared
            // tile, after the rows of the stage are ready and on their way to the peer)
            mbar_init(full_a(s), 2 * ((share ? 1 : kProdWarps) + 1));
            mbar_init(empty_bar(s), share ? 2 : 1);  // both CTAs' MMAs when the tile is shared
        }
        for (int s = 0; s < NS; ++s) mbar_init(rows_ready(s), kProdWarps / 2);   // the group that builds it
        for (int s = 0; s < kInSlots; ++s) {
            mbar_init(full_in(s), 1);
            mbar_init(empty_in(s), share ? kProdWarps / 2 : kProdWarps);
        }
        for (int s = 0; s < NS; s += 2) mbar_init(bfree_first(s), 1);
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, 4 + kProdWarps);   // the epilogue warps and the producer warps
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __shared__ __align__(16) float ref_s[2 * kMaxHalf];           // [2][kMaxHalf]: P_KID, N of the group
    if constexpr (kShare && NJ == 1) {
        const FusedJob& J0 = L.job[0];
        const int cb = static_cast<int>(rank) * J0.F.n_half;       // this CTA's channel group
        for (int c = threadIdx.x; c < kMaxHalf; c += blockDim.x) {
            const bool in = c < J0.F.n_half && cb + c < J0.T.n_ch;
            ref_s[c] = in ? J0.T.ref_pk[cb + c] : 0.f;
            ref_s[kMaxHalf + c] = in ? J0.T.ref_n[cb + c] : 0.f;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (share) cluster_sync_all();              // the peer's barriers exist before any remote arrival
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const uint32_t d_sig = tmem_base;            // columns [0, n_half)
    const uint32_t d_noi = tmem_base + 256;      // columns [256, 256 + n_half)
    unsigned int* const status0 = L.job[0].T.status;   // a wait that runs out marks every job (teardown)

    // Work units: tiles shared by a cluster, or (tile, group) items for independent CTAs.
    const long long n_units = share ? L.n_items / 2 : L.n_items;
    const long long ubase = share ? blockIdx.x / 2 : blockIdx.x;
    const long long ustride = share ? gridDim.x / 2 : gridDim.x;
    const long long my_items = n_units > ubase ? (n_units - ubase + ustride - 1) / ustride : 0;
    auto item_of = [&](long long j) {
        const long long u = ubase + j * ustride;
        return share ? u * 2 + rank : u;
    };
    // The job of launch item it (jobs hold whole tiles, so both items of a shared tile are in one).
    auto job_of = [&](long long it) -> const FusedJob& {
        int k = 0;
        if constexpr (NJ > 1)
            while (k + 1 < L.n_jobs && it >= L.job[k + 1].item0) ++k;
        return L.job[k];
    };

    // ---------------- epilogue of one item: this warp's share of the units ----------------
    // A warp reads the TMEM lanes of its quadrant (warp mod 4) = tile rows [32 quad, 32 quad + 32).
    // Unit u = (chunk u / 4 of 16 channels, 16-lane half (u / 2) % 2, 8-channel group u % 2).  Each
    // quadrant's chunks are split over three warps (the epilogue warp and one warp of each producer
    // group, idle while the accumulators drain) in runs of whole chunks.  (Runs weighted by the cost
    // of drawing normals in the epilogue measured slower: the time per unit is not set by the draw.)
    constexpr int kZChunks = 10;
    static_assert(kZChunks * 16 == 2 * (256 - kMaxHalf), "parked normals fill the columns [176, 256) and [432, 512)");
    const int epi_role = warp >= kEpiWarp0 ? 0 : (warp < kProdWarp0 + 4 ? 1 : 2);
    // This warp's units of an item of job J (they depend on the job's group width and noise flags).
    struct Split {
        int unit_lo, unit_hi, zu_all, n_zunits;
        bool white;
    };
    auto split_of = [&](const FusedJob& J) {
        Split q;
        const int n_chunks = J.F.n_half / 16;
        q.white = (J.T.noise_flags & GATEAU_NOISE_WHITE) != 0;
        const int cut1 = (n_chunks + 2) / 3, cut2 = cut1 + (n_chunks - cut1 + 1) / 2;
        q.unit_lo = 4 * (epi_role == 0 ? 0 : (epi_role == 1 ? cut1 : cut2));
        q.unit_hi = 4 * (epi_role == 0 ? cut1 : (epi_role == 1 ? cut2 : n_chunks));
        q.zu_all = q.white ? 4 * min(n_chunks, kZChunks) : 0;              // units with parked normals
        const int zu_hi = q.white ? min(q.unit_hi, q.zu_all) : q.unit_lo;   // parked units [unit_lo, zu_hi)
        q.n_zunits = zu_hi > q.unit_lo ? zu_hi - q.unit_lo : 0;
        return q;
    };
    const int lq = lane & 3, lr = lane >> 2;
    const bool odd = (lane & 1) != 0;
    // White normals of Eq. 19 for rows (R0, R0 + 8) x channel pairs (chq, chq + 1) of this thread,
    // tile row R0 at sample trow0: a quad's Philox draw serves two lanes (the two channel pairs of
    // the quad); lanes l and l ^ 1 draw it for rows R0 and R0 + 8 respectively and swap the halves
    // the other needs.  Warp-collective (shuffles).
    auto white_pair = [&](const FusedJob& J, long long trow0, int pix, int chq, float2& z0, float2& z1) {
        const float4 z = white_normals4_fast(trow0 + (odd ? 8 : 0), pix, chq >> 2, J.T.key0, J.T.key1);
        const float sx = odd ? z.x : z.z, sy = odd ? z.y : z.w;     // what the partner needs
        const float rx = __shfl_xor_sync(0xffffffffu, sx, 1);
        const float ry = __shfl_xor_sync(0xffffffffu, sy, 1);
        z0 = odd ? make_float2(rx, ry) : make_float2(z.x, z.y);
        z1 = odd ? make_float2(z.z, z.w) : make_float2(rx, ry);
    };
    // The normals depend on (sample, spaxel, channel) only, so the warps that share an item's
    // epilogue draw them for their own units while the item's MMAs run and park them in the TMEM
    // columns the accumulators leave free, [176, 256) and [432, 512): chunks 0..9 of a group, 16
    // columns each (a group's chunk 10 is drawn in the epilogue).  A unit is stored with the shape
    // the epilogue loads it with.
    auto zcol = [](int k) -> uint32_t { return k < 5 ? 176u + 16u * k : 432u + 16u * (k - 5); };
    auto park_unit = [&](const FusedJob& J, const Split& q, int k, long long row0, int pix, int ch_base) {
        const int u = q.unit_lo + k, ck = u >> 2, h = (u >> 1) & 1, g = u & 1, tq = warp & 3;
        float2 z0, z1;
        white_pair(J, J.t0 + row0 + tq * 32 + 16 * h + lr, pix, ch_base + 16 * ck + 8 * g + 2 * lq, z0, z1);
        const float zv[4] = {z0.x, z0.y, z1.x, z1.y};
        tmem_st16x256b_x1(tmem_base + zcol(ck) + 8 * g + (static_cast<uint32_t>(tq * 32 + 16 * h) << 16), zv);
    };
    auto epilogue_item = [&](long long j) -> bool {
        // tcgen05.ld is warp-collective: take the wait's outcome warp-uniformly.
        tmem_wait_st();                          // this warp's parked normals of item j have landed
        const bool okw = mbar_wait(acc_full, static_cast<uint32_t>(j & 1), abort_flag, status0, L.wait_cycles);
        if (!__all_sync(0xffffffffu, okw)) return false;
        tc_fence_after();
        const int quad = warp & 3;
        const int r = quad * 32 + lane;
        const long long it = item_of(j);
        const FusedJob& J = job_of(it);
        const DevTables& T = J.T;
        const Split q = split_of(J);
        const bool white = q.white;
        const int zu_all = q.zu_all;
        long long tile, row0;
        int pix, nrows, grp;
        item_coords(J, it - J.item0, tile, pix, row0, nrows, grp);
        const int ch_base = grp * J.F.n_half;
        // Each 16-lane half of the quadrant is read with the 16x256b shape: a thread holds rows R0
        // and R0 + 8 for channel pairs 2 (lane % 4) + {0, 1} of both 8-channel groups of the chunk,
        // so one store instruction covers 8 rows x 16 contiguous bytes (the 32x32b shape, one row
        // per lane, scattered each store over 32 rows).
        (void)r;
        const long long S_row = static_cast<long long>(T.n_pix) * T.n_ch;
        float* obase = J.out + (row0 * T.n_pix + pix) * static_cast<long long>(T.n_ch);
        // Unit u = (chunk u / 4, half (u / 2) % 2, 8-channel group u % 2): one 16x256b load of each
        // of S, N and the parked normals (a thread: rows R0 and R0 + 8 x channels chq, chq + 1).
        // TMEM reads run one unit ahead: the loads of unit u + 1 are issued before unit u is
        // computed, and each wait names the registers it completes (no use can move above it).
        auto issue = [&](int u, uint32_t (&sr)[4], uint32_t (&nr)[4], uint32_t (&zr)[4]) {
            const int ck = u >> 2;
            const uint32_t lanes = static_cast<uint32_t>(quad * 32 + 16 * ((u >> 1) & 1)) << 16;
            const uint32_t col = 16 * ck + 8 * (u & 1);
            tmem_ld16x256b_x1(d_sig + lanes + col, sr);
            tmem_ld16x256b_x1(d_noi + lanes + col, nr);
            if (white && u < zu_all) tmem_ld16x256b_x1(tmem_base + zcol(ck) + 8 * (u & 1) + lanes, zr);   // warp-uniform
        };
        auto finish = [&](int u, const uint32_t (&sr)[4], const uint32_t (&nr)[4], const uint32_t (&zr)[4]) {
            const int ck = u >> 2, h = (u >> 1) & 1, g = u & 1;
            const int R0 = quad * 32 + 16 * h + lr;                     // tile rows R0, R0 + 8
            const int chq = ch_base + 16 * ck + 8 * g + 2 * lq;         // this thread's channel pair
            float2 z0 = make_float2(0.f, 0.f), z1 = make_float2(0.f, 0.f);   // rows R0, R0 + 8
            if (white && u < zu_all) {
                z0 = make_float2(__uint_as_float(zr[0]), __uint_as_float(zr[1]));
                z1 = make_float2(__uint_as_float(zr[2]), __uint_as_float(zr[3]));
            } else if (white) {
                white_pair(J, J.t0 + row0 + R0, pix, chq, z0, z1);
            }
            // output scale: brightness temperature a P + b (Sect. 2.7), or W (a = 1, b = 0)
            float2 ka = make_float2(1.f, 1.f), kb = make_float2(0.f, 0.f);
            if (T.tb_a && chq < T.n_ch) {
                ka = *reinterpret_cast<const float2*>(T.tb_a + chq);   // padded arrays, chq even
                kb = *reinterpret_cast<const float2*>(T.tb_b + chq);
            }
            // the reference spectrum's P_KID and N (padded to n_ch_pad, chq even): from shared memory
            // in a single-job launch of shared tiles, else from global memory
            float2 rpk = make_float2(0.f, 0.f), rn = make_float2(0.f, 0.f);
            if constexpr (kShare && NJ == 1) {
                const int cl = chq - ch_base;                            // even, < kMaxHalf
                rpk = *reinterpret_cast<const float2*>(ref_s + cl);
                rn = *reinterpret_cast<const float2*>(ref_s + kMaxHalf + cl);
            } else if (chq < T.n_ch) {
                rpk = *reinterpret_cast<const float2*>(T.ref_pk + chq);
                rn = *reinterpret_cast<const float2*>(T.ref_n + chq);
            }
            // The four outputs (rows R0, R0 + 8 x channels chq, chq + 1) are formed without branches,
            // so their dependent chains (the square root on the special-function unit among them)
            // overlap; only the stores are guarded (a ragged last tile, channels past n_ch).
            float v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int rr = k >> 1, e = k & 1;
                const float2 zz = rr ? z1 : z0;
                const float pk = fmaf(T.kb1e9, __uint_as_float(sr[k]), e ? rpk.y : rpk.x);
                // k_B outside the root: k_B^2 times N would leave the normal float range
                const float nn = __uint_as_float(nr[k]) + (e ? rn.y : rn.x);
                const float sigma = T.kB * sqrt_approx(T.noise_scale * fmaxf(nn, 0.f));
                v[k] = fmaf(e ? ka.y : ka.x, fmaf(sigma, e ? zz.y : zz.x, pk), e ? kb.y : kb.x);
            }
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int R = R0 + 8 * rr;
                if (R < nrows) {
                    float* orow = obase + R * S_row;
                    if (chq < T.n_ch) orow[chq] = v[2 * rr];
                    if (chq + 1 < T.n_ch) orow[chq + 1] = v[2 * rr + 1];
                }
            }
        };
        uint32_t sa[4], na[4], za[4] = {0u, 0u, 0u, 0u}, sb[4], nb[4], zb[4] = {0u, 0u, 0u, 0u};
        const int u_end = q.unit_hi;
        int u = q.unit_lo;
        if (u < u_end) issue(u, sa, na, za);
        while (u < u_end) {
            tmem_wait_ld_regs(sa, na, za);
            if (u + 1 < u_end) issue(u + 1, sb, nb, zb);
            finish(u, sa, na, za);
            if (++u >= u_end) break;
            tmem_wait_ld_regs(sb, nb, zb);
            if (u + 1 < u_end) issue(u + 1, sa, na, za);
            finish(u, sb, nb, zb);
            ++u;
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty);   // one arrival per epilogue-sharing warp
        return true;
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- filter operands: one bulk copy per stage (B ring) ----------------
            // Stage g's operands go to B slot g mod NSB and complete on the stage-full barrier of
            // A slot g mod NS.  B slot g mod NSB is free once the MMAs of stage g - NSB are done:
            // for the first stage of a pair its own commit reports it, for the second the commit
            // that frees the pair's A slots.
            // NSB <= NS: the copy for stage g starts after the MMAs of stage g - NSB, so the
            // stage-full barrier is already in stage g's phase.
            long long g = 0;
            int s = 0, sa = 0;
            int sf = 0;                // A slot of stage g - NSB
            uint32_t pf = 0;           // its pass parity over the A ring
            for (long long j = 0; j < my_items && !*abort_flag; ++j) {
                const long long it = item_of(j);
                const FusedJob& J = job_of(it);
                const int n_ks = J.T.Kp / kKStage;
                const int grp = static_cast<int>((it - J.item0) % J.F.n_groups);
                const uint16_t* src = J.F.B + static_cast<size_t>(grp) * n_ks * J.F.stage_elems;
                // this job's operands of a stage (its group width; the slot is sized for the widest)
                const uint32_t bytes = static_cast<uint32_t>(kBMats * J.F.n_half * kKStage * 2);
                // a shared tile also receives the peer's half of the rows (3 matrices x 64 rows x 16 points)
                const uint32_t expect = bytes + (share ? static_cast<uint32_t>(kAMats * kTileM * kKStage) : 0u);
                bool ok = true;
                for (int ks = 0; ks < n_ks; ++ks) {
                    // the copy's addresses are formed before the wait for its slot
                    const uint32_t dst = smem_u32(smem + sp.b_off + s * sp.b_bytes);
                    const uint16_t* op = src + ks * J.F.stage_elems;
                    const uint32_t bar = full_a(sa);
                    if (g >= NSB) {
                        if (!mbar_wait_poll((sf & 1) ? empty_bar(sf) : bfree_first(sf), pf, abort_flag, status0, L.wait_cycles)) {
                            ok = false;
                            break;
                        }
                        if (++sf == NS) { sf = 0; pf ^= 1u; }
                    }
                    mbar_arrive_expect_tx(bar, expect);
                    bulk_g2s(dst, op, bytes, bar);
                    ++g;
                    if (++s == NSB) s = 0;
                    if (++sa == NS) sa = 0;
                }
                if (!ok) break;
            }
            for (long long q = (g > NSB ? g - NSB : 0); q < g; ++q) {   // no copy in flight at exit
                if ((q & 1) == 0 && q + 1 < g) continue;   // stages 2p, 2p + 1 share one barrier phase
                mbar_drain(full_a(static_cast<int>(q % NS)), static_cast<uint32_t>((q / NS) & 1));
            }
        }
    } else if (warp == 2) {
        if (lane == 0) {
            // ---------------- staged gathers: opacity rows + cube box per stage (input ring) ----------------
            long long g = 0;
            int s = 0;
            uint32_t ph = 0;
            for (long long j = 0; j < my_items && !*abort_flag; ++j) {
                const long long it = item_of(j);
                const FusedJob& J = job_of(it);
                const int n_ks = J.T.Kp / kKStage;
                long long tile, row0;
                int pix, nrows, grp;
                item_coords(J, it - J.item0, tile, pix, row0, nrows, grp);
                const TileInfo ti = J.tiles[tile];
                const bool tau_box = J.F.tma_inputs && (ti.flags & TILE_TAU_FITS);
                const bool cube_box = J.F.tma_inputs && (ti.flags & TILE_CUBE_FITS);
                const bool small = (ti.flags & TILE_CUBE_SMALL) != 0;   // the tile's rows stay in one cell row
                const bool tsmall = (ti.flags & TILE_TAU_SMALL) != 0;   // and span one or two opacity rows
                const uint32_t bytes = kConstBytes + (tau_box ? (tsmall ? kTauBoxBytesS : kTauBoxBytes) : 0) +
                                       (cube_box ? (small ? kCubeBoxBytesS : kCubeBoxBytes) : 0);
                bool ok = true;
                for (int ks = 0; ks < n_ks; ++ks) {
                    if (g >= kInSlots && !mbar_wait(empty_in(s), ph ^ 1u, abort_flag, status0, L.wait_cycles)) {
                        ok = false;
                        break;
                    }
                    uint8_t* slot = smem + sp.in_off + static_cast<size_t>(s) * kInSlotBytes;
                    mbar_arrive_expect_tx(full_in(s), bytes);
                    bulk_g2s(smem_u32(slot + kConstOff), J.F.c_tiled + static_cast<size_t>(ks) * 2 * kKStage,
                             kConstBytes, full_in(s));
                    if (cube_box)
                        tensor3d_g2s(smem_u32(slot), small ? &J.tm_cube_s : &J.tm_cube, ks * kKStage, ti.ie0, ti.ia0,
                                     full_in(s));
                    if (tau_box)
                        tensor2d_g2s(smem_u32(slot + kTauOff), tsmall ? &J.tm_tau_s : &J.tm_tau, ks * kKStage, 2 * ti.j0,
                                     full_in(s));
                    ++g;
                    if (++s == kInSlots) { s = 0; ph ^= 1u; }
                }
                if (!ok) break;
            }
            for (long long q = (g > kInSlots ? g - kInSlots : 0); q < g; ++q)
                mbar_drain(full_in(static_cast<int>(q % kInSlots)), static_cast<uint32_t>((q / kInSlots) & 1));
        }
    } else if (warp == 3) {
        // ---------------- shared tiles: this CTA's rows of each stage -> the peer ----------------
        // Off the producers' critical path: they signal rows_ready and go on; this thread issues
        // the three 2 KB bulk copies (its 64 rows of D_hi, D_lo, bf16(D_hi^2)) into the peer's
        // shared memory, completing on the peer's stage-full barrier, then arrives on ours.
        if (share && lane == 0) {
            constexpr uint32_t amat = kTileM * kKStage * 2;
            const uint32_t peer = rank ^ 1u;
            int s = 0;
            uint32_t par = 0;
            bool ok = true;
            for (long long j = 0; j < my_items && ok; ++j) {
                const int n_ks = job_of(item_of(j)).T.Kp / kKStage;
                for (int ks = 0; ks < n_ks; ++ks) {
                    if (!mbar_wait(rows_ready(s), par, abort_flag, status0, L.wait_cycles)) {
                        ok = false;
                        break;
                    }
                    const uint32_t a0 = smem_u32(smem + s * sp.a_bytes);
                    const uint32_t bar_peer = mapa_peer(full_a(s), peer);
#pragma unroll
                    for (int m = 0; m < kAMats; ++m) {
                        const uint32_t src = a0 + m * amat + rank * (amat / 2);
                        bulk_s2peer(mapa_peer(src, peer), src, amat / 2, bar_peer);
                    }
                    mbar_arrive(full_a(s));
                    if (++s == NS) { s = 0; par ^= 1u; }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            // slot-0 descriptors and the per-slot steps of the start-address field
            const uint32_t a_mat = kTileM * kKStage * 2;                // bytes per A matrix
            const uint32_t a_base = smem_u32(smem), b_base = smem_u32(smem + sp.b_off);
            // descriptor low words of slot 0 (start address, leading byte offset) and the common high word
            const uint32_t dx0 = static_cast<uint32_t>(smem_desc(a_base + 0 * a_mat, 128, 256)),
                           dx1 = static_cast<uint32_t>(smem_desc(a_base + 1 * a_mat, 128, 256)),
                           dx2 = static_cast<uint32_t>(smem_desc(a_base + 2 * a_mat, 128, 256));
            const uint32_t dhi = static_cast<uint32_t>(smem_desc(a_base, 128, 256) >> 32);
            const uint32_t a_step = static_cast<uint32_t>(sp.a_bytes >> 4), b_step = static_cast<uint32_t>(sp.b_bytes >> 4);
            int s = 0, sb = 0;
            uint32_t par = 0;
            long long n_pairs = 0;                                     // stage pairs committed
            bool ok = true;
            for (long long j = 0; j < my_items && ok; ++j) {
                // the item's job: its group width sets N and where the B matrices sit in a slot
                const FusedJob& J = job_of(item_of(j));
                const int n_ks = J.T.Kp / kKStage;
                const uint32_t idesc = make_idesc(J.F.n_half);
                const uint32_t b_mat = static_cast<uint32_t>(J.F.n_half) * kKStage * 2;
                const uint32_t dh0 = static_cast<uint32_t>(smem_desc(b_base + 0 * b_mat, 128, 256)),
                               dh1 = static_cast<uint32_t>(smem_desc(b_base + 1 * b_mat, 128, 256)),
                               dh2 = static_cast<uint32_t>(smem_desc(b_base + 2 * b_mat, 128, 256)),
                               dh3 = static_cast<uint32_t>(smem_desc(b_base + 3 * b_mat, 128, 256));
                if (j > 0) {
                    ok = mbar_wait(acc_empty, static_cast<uint32_t>((j - 1) & 1), abort_flag, status0, L.wait_cycles);
                    if (!ok) break;
                    tc_fence_after();
                }
                for (int ks = 0; ks < n_ks; ks += 2) {               // n_ks is even (Kp % 32 == 0)
                    // What the pair's MMAs and commits need is formed before the wait, so that they
                    // go out as soon as the stage data are in.  Descriptors of A slots s, s + 1 and
                    // B slots sb, sb1: the slot-0 low words plus the slot offset in 16-byte units
                    // (start-address field, bits 0-13; no carry: shared addresses stay below 256 KB).
                    const int sb1 = sb + 1 == NSB ? 0 : sb + 1;
                    const uint32_t da0 = static_cast<uint32_t>(s) * a_step, da1 = da0 + a_step;
                    const uint32_t db0 = static_cast<uint32_t>(sb) * b_step, db1 = static_cast<uint32_t>(sb1) * b_step;
                    const uint32_t bar_full = full_a(s), bar_first = bfree_first(s), bar_free = empty_bar(s);
                    const uint32_t acc0 = ks > 0 ? 1u : 0u;
                    if (!mbar_wait_poll(bar_full, par, abort_flag, status0, L.wait_cycles)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    tc_mma_stage(d_sig, d_noi, dx0 + da0, dx1 + da0, dx2 + da0, dh0 + db0, dh1 + db0, dh2 + db0,
                                 dh3 + db0, dhi, idesc, acc0);
                    tc_commit(bar_first);                      // the first stage's B slot
                    tc_mma_stage(d_sig, d_noi, dx0 + da1, dx1 + da1, dx2 + da1, dh0 + db1, dh1 + db1, dh2 + db1,
                                 dh3 + db1, dhi, idesc, 1u);
                    if (share) tc_commit_pair(bar_free);       // A slots s, s+1 free in both CTAs
                    else tc_commit(bar_free);                  // A slots s, s+1 free once these MMAs finish
                    sb = sb1 + 1 == NSB ? 0 : sb1 + 1;
                    s += 2;
                    ++n_pairs;
                    if (s == NS) { s = 0; par ^= 1u; }
                }
                if (!ok) break;
                tc_commit(acc_full);                  // accumulators of item j complete
            }
            tc_commit(drain_bar);                     // no MMA in flight at exit (bounded)
            mbar_drain(drain_bar, 0);
            // A shared tile's stage-free barriers also take the peer's commits, which travel over
            // the cluster; nothing else waits for those of the last pairs.  Waiting here for each
            // of the last pairs to complete (both commits in) leaves no arrival addressed to this
            // CTA in flight when the cluster leaves.
            // The first-stage B commits of the last pairs likewise: nothing else waits for them.
            for (long long q = (n_pairs > NS / 2 ? n_pairs - NS / 2 : 0); q < n_pairs; ++q) {
                const int sq = static_cast<int>((2 * q) % NS);
                const uint32_t pq = static_cast<uint32_t>(((2 * q) / NS) & 1);
                if (share) mbar_drain(empty_bar(sq), pq);
                mbar_drain(bfree_first(sq), pq);
            }
        }
    } else if (warp >= kProdWarp0 && (share || warp < kEpiWarp0)) {
        // ---------------- spectrum producers ----------------
        // Warp = 16 rows x the 16 points of a stage; thread = two rows (r, r + 8: the same place
        // in the warp's two 8-row core-matrix groups) x one quad of 4 points.  Lanes 8q..8q+7 are
        // the 8 rows of quad q, so a quarter-warp phase of a 16-byte shared load reads one quad of
        // (mostly) one table row or texel and broadcasts it.  When the two rows of a thread use the
        // same table row and cube cell (the usual case: samples 50 ms apart) the gathers are read
        // once for both.  A warp's 8-byte stores of one (row, matrix) cover whole core-matrix rows
        // (two wavefronts per 256 bytes).
        // Shared tile: this CTA builds rows [64 rank, 64 rank + 64); three groups of four warps
        // (warps 4-15: the epilogue warps build too) take stages in turn (global stage
        // g = item * n_ks + ks, group = g mod 3), so a warp has three stage periods for one stage;
        // the copier warp ships the stage's rows to the peer once the group has built them.
        // Independent CTA: warps 4-11 build every stage, 16 rows each.
        const int pw = warp - kProdWarp0;
        const int pgrp = share ? pw >> 2 : 0;        // stage residue mod kStep built by this warp
        constexpr int kStep = share ? 3 : 1;         // stages from one of this warp's stages to the next
        const int row_lo = share ? static_cast<int>(rank) * 64 + 16 * (pw & 3) : 16 * pw;   // pw & 3: warp in group
        const int quad = lane >> 3;                  // points 4 quad .. 4 quad + 3 of the stage
        const int rr[2] = {row_lo + (lane & 7), row_lo + (lane & 7) + 8};
        constexpr int amat = kTileM * kKStage * 2;
        enum { kHasSrc = 1, kTauBox = 2, kCubeBox = 4 };
        struct RowC {
            int flags, tau_j, src_idx, sA, sC00;     // staged offsets in floats, without the quad
            float w00, w10, w01, w11, ea, eb;
        };
        long long g = pgrp;                          // this CTA's stage index over its items
        int s = pgrp % NS, si = pgrp % kInSlots;
        uint32_t ph = 0, phi = 0;
        bool ok = true;
        // Item j's first kPre stages are built before the epilogue of item j - 1 (their slots are
        // freed by item j - 1's MMAs alone, kPre <= NS), so the MMAs of item j start as soon as
        // the accumulators drain.  Parked normals of item j: once the epilogue of item j - 1 has
        // read its own, one slice every kZEvery stages after kZSkip stages.
        const int kPre = NS;
        constexpr int kZSkip = 2, kZEvery = share ? 3 : 8;
        RowC rc[2];
        bool same_tau = false, same_cube = false;
        int cstride = kCubeBoxEl * kBoxW;            // floats from a staged texel to its azimuth neighbour (the tile's box)
        long long z_row0 = 0;
        int z_pix = 0, z_chb = 0;
        const FusedJob* Jp = &L.job[0];              // the job of the item being built
        // row constants of item j (and the coordinates its parked normals need)
        auto row_consts = [&](long long j) {
            {
                const long long it = item_of(j);
                const FusedJob& J = job_of(it);
                Jp = &J;
                const DevTables& T = J.T;
                long long tile, row0;
                int pix, nrows, grp;
                item_coords(J, it - J.item0, tile, pix, row0, nrows, grp);
                z_row0 = row0;
                z_pix = pix;
                z_chb = grp * J.F.n_half;
                const TileInfo ti = J.tiles[tile];
                const int box_el = (ti.flags & TILE_CUBE_SMALL) ? kCubeBoxElS : kCubeBoxEl;
                cstride = box_el * kBoxW;
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int r = rr[i];
                    const bool valid = r < nrows;
                    RowParams rp;
                    if (valid) {
                        rp = J.rows[static_cast<long long>(pix) * J.nt + row0 + r];
                    } else {
                        rp.csc = 1.f; rp.tau_j = ti.j0; rp.tau_f = 0.f; rp.src_idx = -1; rp.src_fa = 0.f;
                        rp.src_fe = 0.f; rp.src_cell = -1;
                    }
                    if (rp.tau_j < 0 || rp.tau_j > T.n_pwv - 2) {
                        atomicOr(T.status, GATEAU_STATUS_BAD_INDEX);
                        rp.tau_j = 0;
                    }
                    const bool has_src = valid && rp.src_idx >= 0;
                    // staged boxes, with a range check that sends a row to the global path otherwise
                    const int dj = rp.tau_j - ti.j0;
                    const bool tau_box = J.F.tma_inputs && (ti.flags & TILE_TAU_FITS) && dj >= 0 &&
                                         dj <= ((ti.flags & TILE_TAU_SMALL) ? kTauBoxRowsS : kTauBoxRows) - 1;
                    const int da = has_src ? (rp.src_cell >> 16) - ti.ia0 : 0;
                    const int de = has_src ? (rp.src_cell & 0xffff) - ti.ie0 : 0;
                    const bool cube_box = has_src && J.F.tma_inputs && (ti.flags & TILE_CUBE_FITS) && da >= 0 &&
                                          da <= kCubeBoxAz - 2 && de >= 0 && de <= box_el - 2;
                    RowC& c = rc[i];
                    c.flags = (has_src ? kHasSrc : 0) | (tau_box ? kTauBox : 0) | (cube_box ? kCubeBox : 0);
                    c.tau_j = rp.tau_j;
                    c.src_idx = has_src ? rp.src_idx : 0;
                    c.sA = 2 * dj * kBoxW;
                    c.sC00 = (da * box_el + de) * kBoxW;
                    const float fa = rp.src_fa, fe = rp.src_fe;
                    c.w00 = (1.f - fa) * (1.f - fe); c.w10 = fa * (1.f - fe); c.w01 = (1.f - fa) * fe; c.w11 = fa * fe;
                    // eta_atm = exp(-csc tau) = 2^(a tau_j + b dtau_j) with a = -csc log2(e), b = a f
                    c.ea = -rp.csc * 1.4426950408889634f;
                    c.eb = c.ea * rp.tau_f;
                }
            }
            // the two rows read the same opacity gathers (same table row and path) and / or the
            // same cube gathers (same cell and path)
            same_tau = (rc[0].flags & kTauBox) == (rc[1].flags & kTauBox) && rc[0].tau_j == rc[1].tau_j &&
                       rc[0].sA == rc[1].sA;
            same_cube = (rc[0].flags & (kCubeBox | kHasSrc)) == (rc[1].flags & (kCubeBox | kHasSrc)) &&
                        rc[0].src_idx == rc[1].src_idx && rc[0].sC00 == rc[1].sC00;
        };
        // one stage of this warp (ks of the current item): gathers, X, split, stores, arrival
        auto build_stage = [&](int ks) -> bool {
                bool okw = (g < NS || mbar_wait(empty_bar(s), ph ^ 1u, abort_flag, status0, L.wait_cycles)) &&
                           mbar_wait(full_in(si), phi, abort_flag, status0, L.wait_cycles);
                okw = __all_sync(0xffffffffu, okw);      // the warp signals as one
                if (!okw) return false;
                uint8_t* a0 = smem + s * sp.a_bytes;
                float x[2][4];
                {
                    const float* slot =
                        reinterpret_cast<const float*>(smem + sp.in_off + static_cast<size_t>(si) * kInSlotBytes);
                    const float* stau = slot + kTauOff / 4;
                    const float* scon = slot + kConstOff / 4;                // [c_ref][16], [c1][16]
                    const int kq = ks * kKStage + 4 * quad;                  // first point of this thread
                    const float4 cr = ld4(scon + 4 * quad);
                    const float4 c1 = ld4(scon + kKStage + 4 * quad);
                    float4 ta, td, q00, q10, q01, q11;
                    auto gather_tau = [&](const RowC& c) {
                        if (c.flags & kTauBox) {
                            ta = ld4(stau + c.sA + 4 * quad);
                            td = ld4(stau + c.sA + kBoxW + 4 * quad);
                        } else {
                            const DevTables& T = Jp->T;
                            const float* gA = T.tau + static_cast<long long>(2 * c.tau_j) * T.Kp;
                            ta = ld4(gA + kq);
                            td = ld4(gA + T.Kp + kq);
                        }
                    };
                    auto gather_cube = [&](const RowC& c) {
                        if (c.flags & kCubeBox) {
                            const float* b = slot + c.sC00 + 4 * quad;
                            q00 = ld4(b);
                            q10 = ld4(b + cstride);
                            q01 = ld4(b + kBoxW);
                            q11 = ld4(b + cstride + kBoxW);
                        } else if (c.flags & kHasSrc) {
                            const DevTables& T = Jp->T;
                            const float* g00 = T.cube + c.src_idx + kq;
                            const float* g10 = g00 + static_cast<long long>(T.n_el) * T.Kp;
                            q00 = ld4(g00);
                            q10 = ld4(g10);
                            q01 = ld4(g00 + T.Kp);
                            q11 = ld4(g10 + T.Kp);
                        } else {
                            q00 = q10 = q01 = q11 = make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                    };
                    // Read everything this stage needs from the input slot, then release the slot so
                    // the next gathers land while this warp computes.  D = (c_ref - c1 e) + e P'_src.
                    float4 arg[2], src[2];
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const RowC& c = rc[i];
                        if (i == 0 || !same_tau) gather_tau(c);
                        if (i == 0 || !same_cube) gather_cube(c);
                        arg[i] = make_float4(fmaf(c.eb, td.x, c.ea * ta.x), fmaf(c.eb, td.y, c.ea * ta.y),
                                             fmaf(c.eb, td.z, c.ea * ta.z), fmaf(c.eb, td.w, c.ea * ta.w));
                        src[i].x = c.w00 * q00.x + c.w10 * q10.x + c.w01 * q01.x + c.w11 * q11.x;
                        src[i].y = c.w00 * q00.y + c.w10 * q10.y + c.w01 * q01.y + c.w11 * q11.y;
                        src[i].z = c.w00 * q00.z + c.w10 * q10.z + c.w01 * q01.z + c.w11 * q11.z;
                        src[i].w = c.w00 * q00.w + c.w10 * q10.w + c.w01 * q01.w + c.w11 * q11.w;
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(empty_in(si));
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const float e0 = ex2_approx(arg[i].x), e1 = ex2_approx(arg[i].y);
                        const float e2 = ex2_approx(arg[i].z), e3 = ex2_approx(arg[i].w);
                        x[i][0] = fmaf(e0, src[i].x, fmaf(-c1.x, e0, cr.x));
                        x[i][1] = fmaf(e1, src[i].y, fmaf(-c1.y, e1, cr.y));
                        x[i][2] = fmaf(e2, src[i].z, fmaf(-c1.z, e2, cr.z));
                        x[i][3] = fmaf(e3, src[i].w, fmaf(-c1.w, e3, cr.w));
                    }
                }
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    uint32_t hi[2], lo[2], sq[2];
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const float xa = x[i][2 * q], xb = x[i][2 * q + 1];
                        const __nv_bfloat162 h2 = __floats2bfloat162_rn(xa, xb);
                        hi[q] = *reinterpret_cast<const uint32_t*>(&h2);
                        lo[q] = pack_bf16(xa - __low2float(h2), xb - __high2float(h2));
                        const __nv_bfloat162 s2 = __hmul2(h2, h2);            // bf16(D_hi^2) for the noise term
                        sq[q] = *reinterpret_cast<const uint32_t*>(&s2);
                    }
                    const size_t off = core_offset(rr[i], 4 * quad, kTileM);  // 8-byte aligned
                    *reinterpret_cast<uint2*>(a0 + 0 * amat + off) = make_uint2(hi[0], hi[1]);
                    *reinterpret_cast<uint2*>(a0 + 1 * amat + off) = make_uint2(lo[0], lo[1]);
                    *reinterpret_cast<uint2*>(a0 + 2 * amat + off) = make_uint2(sq[0], sq[1]);
                }
                fence_proxy_async();                     // our generic stores -> the tensor-core (async) proxy
                __syncwarp();
                if (lane == 0) mbar_arrive(share ? rows_ready(s) : full_a(s));
                // this warp's next stage
                g += kStep;
                s += kStep;
                while (s >= NS) { s -= NS; ph ^= 1u; }
                si += kStep;
                while (si >= kInSlots) { si -= kInSlots; phi ^= 1u; }
                return true;
        };
        long long gbase = 0;                         // this CTA's stages before item j
        for (long long j = 0; j < my_items && ok; ++j) {
            row_consts(j);
            const int n_ks = Jp->T.Kp / kKStage;
            const Split zq = split_of(*Jp);
            const int n_zunits = zq.n_zunits;
            // the stages of item j built by this warp (g advances by kStep, across items too:
            // ks = first ks >= 0 with (gbase + ks) mod kStep == pgrp)
            int ks = share ? static_cast<int>(((pgrp - gbase) % kStep + kStep) % kStep) : 0;
            gbase += n_ks;
            int zk = 0, built = 0;
            if (j > 0) {
                for (; ks < n_ks && ks < kPre; ks += kStep)
                    if (!(ok = build_stage(ks))) break;
                if (!ok) break;
                if (!(ok = epilogue_item(j - 1))) break;
                row_consts(j);                       // formed again: not held across the epilogue
            }
            for (; ks < n_ks; ks += kStep) {
                if (!(ok = build_stage(ks))) break;
                if (zk < n_zunits && built >= kZSkip && (built - kZSkip) % kZEvery == 0)
                    park_unit(*Jp, zq, zk++, z_row0, z_pix, z_chb);
                ++built;
            }
            if (!ok) break;
            while (zk < n_zunits) park_unit(*Jp, zq, zk++, z_row0, z_pix, z_chb);
        }
        if (ok && my_items > 0) ok = epilogue_item(my_items - 1);   // this warp's share of the last epilogue
    } else if (warp >= kEpiWarp0) {
        // ---------------- epilogue warps (independent CTAs; shared tiles use them as producers) ----
        for (long long j = 0; j < my_items; ++j) {
            const long long it = item_of(j);
            const FusedJob& J = job_of(it);
            const Split zq = split_of(J);
            if (zq.n_zunits) {                     // idle while item j's MMAs run: park its normals now
                long long tile, row0;
                int pix, nrows, grp;
                item_coords(J, it - J.item0, tile, pix, row0, nrows, grp);
                for (int k = 0; k < zq.n_zunits; ++k) park_unit(J, zq, k, row0, pix, grp * J.F.n_half);
            }
            if (!epilogue_item(j)) break;
        }
    }

    if (warp >= kProdWarp0) tmem_wait_st();     // no parked normals in flight (a role may have stopped early)
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag)        // a wait ran out: every job of the launch is incomplete
        for (int k = 0; k < L.n_jobs; ++k) atomicOr(L.job[k].T.status, GATEAU_STATUS_WAIT_TIMEOUT);
    if (share && *abort_flag) {                 // aborted shared tile: the row copies already issued land first
        if (threadIdx.x == 0) {
            const long long t_start = clock64();
            while (clock64() - t_start < kAbortGraceCycles) {
            }
        }
        __syncthreads();
    }
    if (share) cluster_sync_all();              // no copy into or out of our shared memory in flight
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
    }
}

// Build the job table of a launch and launch it.  All runs share the launch mode: two channel
// groups each (2-CTA clusters with shared tiles), or any other group count (independent CTAs).
template <int NJ>
static cudaError_t launch_jobs(const FusedRunDesc* runs, int n, int n_sm, cudaStream_t stream) {
    std::unique_ptr<FusedLaunch<NJ>> Lp(new (std::nothrow) FusedLaunch<NJ>());   // ~27 KB: not on the stack
    if (!Lp) return cudaErrorMemoryAllocation;
    FusedLaunch<NJ>& L = *Lp;
    memset(&L, 0, sizeof(L));
    const int share = runs[0].F.n_groups == 2 ? 1 : 0;
    int layout = 16, ring_b = kMaxRingB;
    long long items = 0, wait = kDefaultWaitCycles;
    for (int k = 0; k < n; ++k) {
        const FusedRunDesc& r = runs[k];
        const FusedOperands& F = r.F;
        if (F.n_half < 16 || F.n_half > kMaxHalf || F.n_half % 16 || F.n_kstage % 2 || F.n_kstage * kKStage != r.T.Kp ||
            F.ring_b < 2 || F.ring_b > kMaxRingB ||
            (F.n_groups == 2 ? 1 : 0) != share || F.n_groups < 1 || r.nt < 1 || r.T.n_pix < 1)
            return cudaErrorInvalidConfiguration;
        FusedJob& J = L.job[k];
        memcpy(&J.tm_tau, &r.tm_tau, sizeof(J.tm_tau));
        memcpy(&J.tm_tau_s, &r.tm_tau_s, sizeof(J.tm_tau_s));
        memcpy(&J.tm_cube, &r.tm_cube, sizeof(J.tm_cube));
        memcpy(&J.tm_cube_s, &r.tm_cube_s, sizeof(J.tm_cube_s));
        J.T = r.T;
        J.F = F;
        J.rows = r.rows;
        J.tiles = r.tiles;
        J.t0 = r.t0;
        J.nt = r.nt;
        J.out = r.out;
        J.tiles_per_pix = (r.nt + kTileM - 1) / kTileM;
        J.item0 = items;
        J.n_items = J.tiles_per_pix * r.T.n_pix * F.n_groups;
        items += J.n_items;
        layout = F.n_half > layout ? F.n_half : layout;
        ring_b = F.ring_b < ring_b ? F.ring_b : ring_b;
        wait = F.wait_cycles < wait ? F.wait_cycles : wait;
    }
    L.n_jobs = n;
    L.layout_half = layout;
    L.ring_b = ring_b;
    L.n_items = items;
    L.wait_cycles = wait;
    const SmemPlan sp = smem_plan(layout, ring_b);
    if (!ring_protocol_ok(sp)) return cudaErrorInvalidConfiguration;
    auto kernel = share ? fused_bf16x3_kernel<1, NJ> : fused_bf16x3_kernel<0, NJ>;
    // The kernel's shared-memory limit (set once per kernel and device, to the most any plan takes)
    // and, for clusters, how many fit at this size (queried once per kernel, size and device): a
    // launch is then stream work alone, so a run can be captured into a CUDA graph.
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int max_clusters = 0;
    {
        static std::mutex mu;
        static std::map<std::pair<const void*, int>, bool> limit_set;
        static std::map<std::tuple<const void*, size_t, int>, int> ready;   // -> clusters that fit (0: none)
        std::lock_guard<std::mutex> lk(mu);
        const void* kf = reinterpret_cast<const void*>(kernel);
        if (!limit_set.count(std::make_pair(kf, dev))) {
            static_assert(kMaxSmem <= 227 * 1024, "the fused kernel's shared memory stays within an SM's opt-in limit");
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
            if (e != cudaSuccess) return e;
            limit_set[std::make_pair(kf, dev)] = true;
        }
        const auto key = std::make_tuple(kf, sp.total, dev);
        auto f = ready.find(key);
        if (f == ready.end()) {
            if (share) {
                cudaLaunchConfig_t q = {};
                cudaLaunchAttribute a[1];
                a[0].id = cudaLaunchAttributeClusterDimension;
                a[0].val.clusterDim.x = 2;
                a[0].val.clusterDim.y = 1;
                a[0].val.clusterDim.z = 1;
                q.attrs = a;
                q.numAttrs = 1;
                q.blockDim = dim3(kThreads);
                q.dynamicSmemBytes = sp.total;
                q.gridDim = dim3(static_cast<unsigned>(n_sm / 2 * 2));
                e = cudaOccupancyMaxActiveClusters(&max_clusters, kernel, &q);
                if (e != cudaSuccess) return e;
            }
            f = ready.emplace(key, max_clusters).first;
        }
        max_clusters = f->second;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = sp.total;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    long long grid;
    if (share) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (max_clusters < 1) return cudaErrorInvalidConfiguration;
        const long long tiles = items / 2;
        grid = 2 * (tiles < max_clusters ? tiles : max_clusters);
    } else {
        cfg.attrs = nullptr;
        cfg.numAttrs = 0;
        grid = items < n_sm ? items : n_sm;
    }
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    e = cudaLaunchKernelEx(&cfg, kernel, L);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_fused_runs(const FusedRunDesc* runs, int n, int n_sm, cudaStream_t stream) {
    if (n < 1 || n > kMaxJobs) return cudaErrorInvalidValue;
    return n == 1 ? launch_jobs<1>(runs, n, n_sm, stream) : launch_jobs<kMaxJobs>(runs, n, n_sm, stream);
}

int fused_max_jobs() { return kMaxJobs; }

}  // namespace gateau
