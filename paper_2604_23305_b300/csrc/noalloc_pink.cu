// Allocation-free entry point for the pink-noise scan.
//
// Some callers cannot allocate device memory while they run this library: a
// host process that hands the GPU to an embedding runtime with its own fixed
// memory pool, real-time acquisition loops that forbid cudaMalloc (it can
// synchronise the device and its latency is unbounded), or code running under
// a memory cap where every byte was reserved at start-up.  For them this file
// offers a variant of the pink-noise scan whose scratch memory (the per-chunk
// filter states of the parallel scan) is a file-scope device array, reserved
// when the library is loaded and held by every GPU that loads it until the
// process exits.  The caller passes the filter coefficients, the carried
// state and the output; the call allocates nothing.
#include <mutex>

#include "gateau_internal.h"

namespace gateau {

// Scratch for the chunk states [C][n_pix * n_ch][n_pole]: 1 Mi floats = 4 MiB.
constexpr size_t kNoallocScratchFloats = size_t(1) << 20;
static __device__ __align__(256) float g_pink_scratch[kNoallocScratchFloats];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
float* g_scratch_ptr[kMaxDevices] = {nullptr};

gateau_status noalloc_fail(gateau_status st, const std::string& msg) {
    set_last_error(msg);        // read back with gateau_last_error()
    return st;
}

// Device address of g_pink_scratch on the current device.  In host code the
// array's name is only a stand-in, so the address is looked up once per device
// (with that device current) and cached.
cudaError_t scratch_address(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_pink_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace gateau

using namespace gateau;

extern "C" gateau_status gateau_pink_noise_noalloc(const float* pink_a, const float* pink_r, const float* pink_d,
                                                   int n_pix, int n_ch, int n_pole, unsigned long long seed,
                                                   long long t0, long long nt, float* state, float* out,
                                                   void* stream) {
    if (!pink_a || !pink_r || !pink_d || !state || !out)
        return noalloc_fail(GATEAU_EINVAL, "coefficient, state and output pointers must be non-NULL");
    if (n_pix < 1 || n_ch < 1 || n_pole < 1 || n_pole > kMaxPoles || t0 < 0 || nt < 1)
        return noalloc_fail(GATEAU_EINVAL, "need n_pix, n_ch, nt >= 1, 1 <= n_pole <= 24 and t0 >= 0");
    const long long S = static_cast<long long>(n_pix) * n_ch;
    const long long per_chunk = S * n_pole;
    if (per_chunk > static_cast<long long>(kNoallocScratchFloats))
        return noalloc_fail(GATEAU_EINVAL, "n_pix * n_ch * n_pole = " + std::to_string(per_chunk) +
                                               " exceeds the 1048576 floats of fixed scratch");
    if (nt > (1LL << 31) / n_pix)               // nt * n_pix > 2^31, compared without forming the product
        return noalloc_fail(GATEAU_EINVAL, "nt * n_pix must stay below 2^31");
    float* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess)
        return noalloc_fail(GATEAU_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));

    // Same chunking rule as the allocating path, capped so the chunk states fit the scratch.
    PinkWork W;
    pink_choose_chunks(nt, S, W.C, W.L);
    const long long c_max = static_cast<long long>(kNoallocScratchFloats) / per_chunk;
    if (W.C > c_max) {
        const long long c = c_max < 1 ? 1 : c_max;
        W.L = ((nt + c - 1) / c + 3) / 4 * 4;
        W.C = static_cast<int>((nt + W.L - 1) / W.L);
    }
    W.agg = scratch;            // every chunk state is written by phase 1 before it is read

    DevTables T{};
    T.n_pix = n_pix;
    T.n_ch = n_ch;
    T.n_pole = n_pole;
    T.pink_a = pink_a;
    T.pink_r = pink_r;
    T.pink_d = pink_d;
    T.key0 = static_cast<uint32_t>(seed & 0xffffffffull);
    T.key1 = static_cast<uint32_t>(seed >> 32);
    e = launch_pink(T, state, W, t0, nt, out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return noalloc_fail(GATEAU_ECUDA, std::string("pink launch: ") + cudaGetErrorString(e));
    return GATEAU_OK;
}
