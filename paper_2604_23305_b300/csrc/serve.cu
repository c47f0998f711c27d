// Serving runtime: continuous batching of whole simulations on one GPU.
//
// The paper simulates one observation per call (Sect. 3).  A simulation
// service runs many of them for many users: requests of different spaxel
// counts, channel counts, spectral grids and scan lengths arrive over time.
// This server admits a request when one of its slots and enough of its device
// memory budget are free (first come, first served), creates the request's
// plan then, runs the scan in time chunks on one of its CUDA streams (two
// chunks in flight per request, so the chunks of all admitted requests overlap
// on the GPU), copies every chunk's TOD to pinned host memory, and releases the
// plan when the last chunk is on the host.  Latency = arrival -> last chunk on
// the host; p50/p99 over the requests that completed.
//
// With shared launches the chunks go in rounds instead: a round takes the next
// chunk of every admitted request that has a free chunk buffer and runs them as
// one gateau_run_batch on the server's compute stream, so the requests'
// contractions share persistent launches of the fused kernel (uneven requests
// fill the GPU together); two rounds are in flight, and each request's checksum
// and copy to the host wait for its round on the request's own stream.  The
// persistent launches hold every SM while they run, so the whole round -- row
// setups, shared contractions, noise -- stays on the compute stream.
//
// A dry-run mode replays the same scheduling decisions on a virtual clock with
// no CUDA call, so the admission, slot and budget logic is testable on a host
// without a GPU.  Plans can be built (factory + gateau_plan_prepare: filter
// design, operand tiling, uploads) on builder threads, so an admission does not
// hold up the launches of the requests already running.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gateau_internal.h"

namespace gateau {
namespace {

constexpr int kSumBlocks = 148;        // fixed grid: the checksum's summation order never changes
constexpr int kSumThreads = 256;

// Per-block float64 sums of x and x^2 (grid-stride, fixed order).
__global__ void __launch_bounds__(kSumThreads) tod_partial_sums(const float* __restrict__ x, long long n,
                                                                double* __restrict__ part) {
    double s = 0.0, q = 0.0;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double v = x[i];
        s += v;
        q += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        q += __shfl_down_sync(0xffffffffu, q, o);
    }
    __shared__ double ws[2][kSumThreads / 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        ws[0][w] = s;
        ws[1][w] = q;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int k = 0; k < kSumThreads / 32; ++k) {
            a += ws[0][k];
            c += ws[1][k];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = c;
    }
}

__global__ void tod_sum_parts(const double* __restrict__ part, double* __restrict__ out) {
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int k = 0; k < kSumBlocks; ++k) {
            a += part[2 * k];
            c += part[2 * k + 1];
        }
        out[0] = a;
        out[1] = c;
    }
}

enum { kPending = 0, kActive = 1, kDone = 2, kFailed = 3, kBuilding = 4 };

// Chunks in flight per request: two on the request's own stream; three with shared launches, so
// that a full round can be queued while the copies of the round before last are still running.
constexpr int kMaxDepth = 3;

// Builder threads: create (factory) and prepare the plans of admitted requests.
struct Builders {
    std::mutex mu;
    std::condition_variable cv;
    std::deque<int> todo;
    std::vector<std::pair<int, gateau_plan*>> done;   // plan NULL: the factory or prepare failed
    bool stop = false;
    std::vector<std::thread> threads;
};

struct Slot {
    float* d_out = nullptr;          // chunk TOD (device)
    double* d_part = nullptr;        // per-block checksum parts + final sum (device)
    bool busy = false;
    long long t0 = 0, nt = 0;
    double t_end = 0.0;              // dry run: virtual completion time
};

struct Req {
    gateau_request r{};
    int state = kPending;
    gateau_plan* plan = nullptr;
    size_t held = 0;                 // budget bytes held
    long long chunk = 0;             // samples per chunk
    size_t chunk_bytes = 0;
    long long next_t0 = 0, done_t0 = 0;
    long long launched = 0, retired = 0;   // chunk counters (slot = counter mod the chunk depth)
    int stream = 0, pin = -1;
    Slot slot[kMaxDepth];
    double sum = 0.0, sumsq = 0.0;
    double t_admit = 0.0, t_done = 0.0;
};

// Pinned host staging of one admitted request: two chunk buffers + two checksum pairs.
struct PinPair {
    float* buf[kMaxDepth] = {nullptr, nullptr, nullptr};
    double* sums = nullptr;          // [kMaxDepth][2]
    cudaEvent_t ev[kMaxDepth] = {nullptr, nullptr, nullptr};
};

gateau_status server_fail(gateau_status st, const std::string& msg) {
    set_last_error(msg);
    return st;
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * static_cast<double>(v.size() - 1);
    const size_t i = static_cast<size_t>(std::floor(pos));
    const size_t j = std::min(i + 1, v.size() - 1);
    const double f = pos - static_cast<double>(i);
    return v[i] + f * (v[j] - v[i]);
}

}  // namespace
}  // namespace gateau

using namespace gateau;

struct gateau_server {
    gateau_server_desc d{};
    cudaStream_t batch_stream = nullptr;   // shared launches: the rounds' compute stream
    cudaEvent_t round_ev[2] = {nullptr, nullptr};
    std::vector<cudaStream_t> streams;
    std::vector<PinPair> pins;
    std::vector<int> free_pins;
    std::vector<Req> reqs;           // last run
};

namespace {

void release_slots(Req& q, cudaStream_t st) {
    for (Slot& s : q.slot) {
        if (s.d_out) cudaFreeAsync(s.d_out, st);
        if (s.d_part) cudaFreeAsync(s.d_part, st);
        s = Slot{};
    }
}

}  // namespace

extern "C" {

gateau_status gateau_server_create(const gateau_server_desc* desc, gateau_server** out) {
    if (!desc || !out) return server_fail(GATEAU_EINVAL, "desc and out must be non-NULL");
    *out = nullptr;
    const gateau_server_desc& d = *desc;
    if (d.max_active < 1 || d.max_active > 256) return server_fail(GATEAU_EINVAL, "max_active must be in 1..256");
    if (d.n_streams < 1 || d.n_streams > 256) return server_fail(GATEAU_EINVAL, "n_streams must be in 1..256");
    if (d.chunk_samples < 1) return server_fail(GATEAU_EINVAL, "chunk_samples must be >= 1");
    if (d.max_chunk_bytes < 4096) return server_fail(GATEAU_EINVAL, "max_chunk_bytes must be >= 4096");
    if (d.budget_bytes == 0) return server_fail(GATEAU_EINVAL, "budget_bytes must be > 0");
    if (d.dry_run && !(d.dry_seconds_per_sample >= 0.0))
        return server_fail(GATEAU_EINVAL, "dry_seconds_per_sample must be >= 0");
    const int depth = d.shared_launches ? 3 : 2;   // chunks in flight per request
    if (!d.dry_run && static_cast<double>(d.max_chunk_bytes) * depth * d.max_active > 16.0 * (1ull << 30))
        return server_fail(GATEAU_EINVAL, "pinned staging (2, or 3 with shared launches) x max_active x max_chunk_bytes "
                                          "must stay <= 16 GiB");
    gateau_server* s = new (std::nothrow) gateau_server();
    if (!s) return server_fail(GATEAU_ENOMEM, "host allocation failed");
    s->d = d;
    if (!d.dry_run) {
        cudaError_t e = cudaSuccess;
        // With shared launches the requests' streams (checksums and copies to the host) take
        // priority over the compute stream, so their small kernels get SMs between the rounds.
        int prio_low = 0, prio_high = 0;
        if (d.shared_launches) {
            e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
            if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->batch_stream, cudaStreamNonBlocking, prio_low);
            for (int r = 0; r < 2 && e == cudaSuccess; ++r)
                e = cudaEventCreateWithFlags(&s->round_ev[r], cudaEventDisableTiming);
        }
        for (int i = 0; i < d.n_streams && e == cudaSuccess; ++i) {
            cudaStream_t st = nullptr;
            e = d.shared_launches ? cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio_high)
                                  : cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (e == cudaSuccess) s->streams.push_back(st);
        }
        s->pins.resize(d.max_active);
        for (int i = 0; i < d.max_active && e == cudaSuccess; ++i) {
            PinPair& p = s->pins[i];
            for (int b = 0; b < depth && e == cudaSuccess; ++b) {
                e = cudaHostAlloc(reinterpret_cast<void**>(&p.buf[b]), d.max_chunk_bytes, cudaHostAllocDefault);
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.ev[b], cudaEventDisableTiming);
            }
            if (e == cudaSuccess)
                e = cudaHostAlloc(reinterpret_cast<void**>(&p.sums), 2 * kMaxDepth * sizeof(double), cudaHostAllocDefault);
        }
        if (e != cudaSuccess) {
            gateau_server_destroy(s);
            return server_fail(e == cudaErrorMemoryAllocation ? GATEAU_ENOMEM : GATEAU_ECUDA,
                               std::string("server setup: ") + cudaGetErrorString(e));
        }
    }
    *out = s;
    return GATEAU_OK;
}

void gateau_server_destroy(gateau_server* s) {
    if (!s) return;
    if (s->batch_stream) cudaStreamSynchronize(s->batch_stream);
    for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
    for (PinPair& p : s->pins) {
        for (int b = 0; b < kMaxDepth; ++b) {
            if (p.buf[b]) cudaFreeHost(p.buf[b]);
            if (p.ev[b]) cudaEventDestroy(p.ev[b]);
        }
        if (p.sums) cudaFreeHost(p.sums);
    }
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    for (cudaEvent_t ev : s->round_ev)
        if (ev) cudaEventDestroy(ev);
    if (s->batch_stream) cudaStreamDestroy(s->batch_stream);
    delete s;
}

gateau_status gateau_server_run(gateau_server* srv, const gateau_request* requests, int n,
                                gateau_plan_factory create, gateau_plan_release release, void* user,
                                gateau_server_stats* stats) {
    if (!srv || (!requests && n > 0) || !create || !release)
        return server_fail(GATEAU_EINVAL, "server, requests, create and release must be non-NULL");
    if (n < 0 || n > 1000000) return server_fail(GATEAU_EINVAL, "n must be in 0..1000000");
    for (int i = 0; i < n; ++i) {
        const gateau_request& r = requests[i];
        if (r.nt < 1 || r.n_pix < 1 || r.n_ch < 1 || !(r.arrival_s >= 0.0))
            return server_fail(GATEAU_EINVAL, "request " + std::to_string(i) + ": need nt, n_pix, n_ch >= 1, arrival >= 0");
        if (i > 0 && r.arrival_s < requests[i - 1].arrival_s)
            return server_fail(GATEAU_EINVAL, "arrival times must be non-decreasing");
    }
    const gateau_server_desc& d = srv->d;
    const bool dry = d.dry_run != 0;
    const bool shared = d.shared_launches != 0;
    const int depth = shared ? 3 : 2;                                 // chunks in flight per request
    srv->reqs.assign(n, Req{});
    std::vector<Req>& R = srv->reqs;
    srv->free_pins.clear();
    for (int i = d.max_active - 1; i >= 0; --i) srv->free_pins.push_back(i);
    std::vector<double> stream_free(std::max(d.n_streams, 1), 0.0);   // dry run: virtual stream clocks
    double batch_free = 0.0;                                          // dry run: the compute stream's clock
    long long rounds_launched = 0, rounds_retired = 0, round_members = 0;
    double round_end[2] = {0.0, 0.0};                                 // dry run: virtual round completions

    const auto t_start = std::chrono::steady_clock::now();
    double vclock = 0.0;
    auto now = [&]() {
        if (dry) return vclock;
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    };

    int next = 0, n_active = 0, n_finished = 0, admitted_count = 0;
    size_t held = 0, peak_bytes = 0;
    int peak_active = 0;
    double overlap_sum = 0.0;
    long long overlap_n = 0;
    gateau_status run_status = GATEAU_OK;
    std::string run_error;

    auto finish = [&](Req& q, int idx, int state) {
        if (q.plan) release(user, idx, q.plan);
        q.plan = nullptr;
        if (!dry) {
            cudaStream_t st = srv->streams[q.stream];
            release_slots(q, st);
            if (q.pin >= 0) srv->free_pins.push_back(q.pin);
        }
        q.pin = -1;
        held -= q.held;
        q.held = 0;
        q.state = state;
        q.t_done = now();
        --n_active;
        ++n_finished;
    };

    // An admitted request whose plan exists: a stream, pinned staging and chunk buffers.
    auto activate = [&](Req& q, int idx, gateau_plan* plan) {
        q.plan = plan;
        if (!plan) {                                  // the factory or the preparation failed
            finish(q, idx, kFailed);
            return;
        }
        q.stream = admitted_count % d.n_streams;
        ++admitted_count;
        q.state = kActive;
        if (dry) return;
        q.pin = srv->free_pins.back();
        srv->free_pins.pop_back();
        // with shared launches the chunk buffers are written on the compute stream first
        cudaStream_t st = shared ? srv->batch_stream : srv->streams[q.stream];
        cudaError_t e = cudaSuccess;
        for (int b = 0; b < depth && e == cudaSuccess; ++b) {
            e = cudaMallocAsync(reinterpret_cast<void**>(&q.slot[b].d_out), q.chunk_bytes, st);
            if (e == cudaSuccess)
                e = cudaMallocAsync(reinterpret_cast<void**>(&q.slot[b].d_part), (2 * kSumBlocks + 2) * sizeof(double), st);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            finish(q, idx, kFailed);
        }
    };

    Builders B;
    std::vector<std::pair<int, gateau_plan*>> failed_builds;   // guarded by B.mu
    int n_building = 0;
    const bool use_builders = !dry && d.n_builders > 0;
    if (use_builders) {
        int dev = 0;
        cudaGetDevice(&dev);
        for (int w = 0; w < d.n_builders; ++w)
            B.threads.emplace_back([&, dev]() {
                cudaSetDevice(dev);
                while (true) {
                    int idx = -1;
                    {
                        std::unique_lock<std::mutex> lk(B.mu);
                        B.cv.wait(lk, [&] { return B.stop || !B.todo.empty(); });
                        if (B.todo.empty()) return;           // stop requested and nothing left
                        idx = B.todo.front();
                        B.todo.pop_front();
                    }
                    gateau_plan* plan = create(user, idx);
                    if (plan && gateau_plan_prepare(plan) != GATEAU_OK) {
                        std::lock_guard<std::mutex> lk(B.mu);
                        B.done.emplace_back(idx, plan);      // released by the server thread
                        B.done.back().second = nullptr;
                        failed_builds.push_back(std::make_pair(idx, plan));
                        continue;
                    }
                    std::lock_guard<std::mutex> lk(B.mu);
                    B.done.emplace_back(idx, plan);
                }
            });
    }

    while (n_finished < n) {
        bool progress = false;
        const double t = now();
        // plans whose preparation failed on a builder: hand them back to the caller
        if (use_builders) {
            std::vector<std::pair<int, gateau_plan*>> bad;
            {
                std::lock_guard<std::mutex> lk(B.mu);
                bad.swap(failed_builds);
            }
            for (auto& pr : bad) release(user, pr.first, pr.second);
        }

        // 1. retire chunks whose TOD reached the host (in order per request)
        for (int i = 0; i < n && run_status == GATEAU_OK; ++i) {
            Req& q = R[i];
            if (q.state != kActive) continue;
            while (q.retired < q.launched) {
                Slot& sl = q.slot[q.retired % depth];
                if (dry) {
                    if (sl.t_end > t) break;
                } else {
                    const cudaError_t e = cudaEventQuery(srv->pins[q.pin].ev[q.retired % depth]);
                    if (e == cudaErrorNotReady) break;
                    if (e != cudaSuccess) {
                        run_status = GATEAU_ECUDA;
                        run_error = std::string("chunk completion: ") + cudaGetErrorString(e);
                        break;
                    }
                    const double* cs = srv->pins[q.pin].sums + 2 * (q.retired % depth);
                    q.sum += cs[0];
                    q.sumsq += cs[1];
                    if (q.r.host_out) {
                        const size_t row = static_cast<size_t>(q.r.n_pix) * q.r.n_ch;
                        memcpy(q.r.host_out + static_cast<size_t>(sl.t0) * row, srv->pins[q.pin].buf[q.retired % depth],
                               static_cast<size_t>(sl.nt) * row * sizeof(float));
                    }
                }
                sl.busy = false;
                q.done_t0 += sl.nt;
                ++q.retired;
                progress = true;
            }
            if (run_status != GATEAU_OK) break;
            if (q.done_t0 == q.r.nt) finish(q, i, kDone);
        }
        if (run_status != GATEAU_OK) break;

        // 2. admit arrivals, first come first served
        while (next < n && R[next].state == kPending && requests[next].arrival_s <= now()) {
            Req& q = R[next];
            q.r = requests[next];
            const size_t row_bytes = static_cast<size_t>(q.r.n_pix) * q.r.n_ch * sizeof(float);
            long long chunk = std::min<long long>(d.chunk_samples, q.r.nt);
            chunk = std::min<long long>(chunk, std::max<long long>(1, static_cast<long long>(d.max_chunk_bytes / row_bytes)));
            if (row_bytes > d.max_chunk_bytes) chunk = 0;
            q.chunk = chunk;
            q.chunk_bytes = static_cast<size_t>(chunk) * row_bytes;
            const size_t need = q.r.device_bytes + depth * (q.chunk_bytes + (2 * kSumBlocks + 2) * sizeof(double));
            if (chunk == 0 || need > d.budget_bytes) {   // can never run
                q.state = kFailed;
                q.t_admit = q.t_done = now();
                ++n_finished;
                ++next;
                progress = true;
                continue;
            }
            if (n_active >= d.max_active || held + need > d.budget_bytes) break;   // wait for room
            q.t_admit = now();
            q.held = need;
            held += need;
            peak_bytes = std::max(peak_bytes, held);
            ++n_active;
            peak_active = std::max(peak_active, n_active);
            if (use_builders) {
                q.state = kBuilding;
                ++n_building;
                {
                    std::lock_guard<std::mutex> lk(B.mu);
                    B.todo.push_back(next);
                }
                B.cv.notify_one();
            } else {
                gateau_plan* plan = create(user, next);
                if (plan && !dry && gateau_plan_prepare(plan) != GATEAU_OK) {
                    release(user, next, plan);
                    plan = nullptr;
                }
                activate(q, next, plan);
            }
            ++next;
            progress = true;
        }

        // 2b. plans finished by the builders
        if (use_builders && n_building > 0) {
            std::vector<std::pair<int, gateau_plan*>> ready;
            {
                std::lock_guard<std::mutex> lk(B.mu);
                ready.swap(B.done);
            }
            for (auto& pr : ready) {
                --n_building;
                activate(R[pr.first], pr.first, pr.second);
                progress = true;
            }
        }

        // 3. launch chunks: every active request keeps two in flight
        // The checksum and the copy to the host of a chunk written into slot b of request q, on
        // the request's stream (false: a CUDA error, recorded in run_status).
        auto post_chunk = [&](Req& q, int b, long long len) -> bool {
            cudaStream_t st = srv->streams[q.stream];
            PinPair& pp = srv->pins[q.pin];
            Slot& sl = q.slot[b];
            const long long n_el = len * q.r.n_pix * q.r.n_ch;
            tod_partial_sums<<<kSumBlocks, kSumThreads, 0, st>>>(sl.d_out, n_el, sl.d_part);
            tod_sum_parts<<<1, 32, 0, st>>>(sl.d_part, sl.d_part + 2 * kSumBlocks);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(pp.sums + 2 * b, sl.d_part + 2 * kSumBlocks, 2 * sizeof(double),
                                    cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(pp.buf[b], sl.d_out, static_cast<size_t>(n_el) * sizeof(float),
                                    cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaEventRecord(pp.ev[b], st);
            if (e != cudaSuccess) {
                run_status = GATEAU_ECUDA;
                run_error = std::string("chunk launch: ") + cudaGetErrorString(e);
                return false;
            }
            return true;
        };
        auto count_overlap = [&]() {
            int inflight = 0;
            for (const Req& o : R)
                if (o.state == kActive && o.launched > o.retired) ++inflight;
            overlap_sum += inflight;
            ++overlap_n;
        };
        if (shared) {
            // rounds that finished on the compute stream
            while (rounds_retired < rounds_launched) {
                const int r = static_cast<int>(rounds_retired & 1);
                if (dry) {
                    if (round_end[r] > t) break;
                } else if (cudaEventQuery(srv->round_ev[r]) != cudaSuccess) {
                    break;                         // not ready (or an error that the chunk events report)
                }
                ++rounds_retired;
            }
            // A round: the next chunk of every active request with a free buffer.  A round is formed
            // when none is in flight (the GPU would idle), or when one is in flight and every active
            // request can join (a second, full round queued behind it); so rounds stay whole instead
            // of splitting as the requests' copies to the host finish one by one.
            std::vector<int> members;
            int waiting = 0;
            for (int i = 0; i < n; ++i) {
                const Req& q = R[i];
                if (q.state != kActive || q.next_t0 >= q.r.nt) continue;
                if (q.launched - q.retired < depth) members.push_back(i);
                else ++waiting;
            }
            const long long pending = rounds_launched - rounds_retired;
            if (!(pending == 0 || (pending == 1 && waiting == 0))) members.clear();
            if (!members.empty()) {
                std::vector<gateau_plan*> plans;
                std::vector<long long> t0s, nts;
                std::vector<float*> outs;
                double work = 0.0;
                for (int i : members) {
                    Req& q = R[i];
                    const long long len = std::min(q.chunk, q.r.nt - q.next_t0);
                    plans.push_back(q.plan);
                    t0s.push_back(q.next_t0);
                    nts.push_back(len);
                    outs.push_back(q.slot[q.launched % depth].d_out);
                    work += static_cast<double>(len) * q.r.n_pix * q.r.n_ch * d.dry_seconds_per_sample;
                }
                const int r = static_cast<int>(rounds_launched & 1);
                bool enqueued = true;
                if (dry) {
                    const double start = std::max(now(), batch_free);
                    batch_free = start + work;
                    round_end[r] = batch_free;
                } else {
                    // the whole round on the compute stream (the persistent launches hold every SM,
                    // so the round's own row setup and noise run between them there); round_ev[r]
                    // marks its end, after which each request's checksum and copy follow on its stream
                    gateau_status gs = gateau_run_batch(plans.data(), t0s.data(), nts.data(), outs.data(),
                                                        static_cast<int>(members.size()), srv->batch_stream);
                    if (gs != GATEAU_OK) {                 // nothing of this round was enqueued
                        enqueued = false;
                        cudaStreamSynchronize(srv->batch_stream);
                        for (int i : members) {
                            cudaStreamSynchronize(srv->streams[R[i].stream]);
                            finish(R[i], i, kFailed);
                        }
                        progress = true;
                    } else {
                        cudaError_t e = cudaEventRecord(srv->round_ev[r], srv->batch_stream);
                        for (size_t m = 0; m < members.size() && e == cudaSuccess; ++m)
                            e = cudaStreamWaitEvent(srv->streams[R[members[m]].stream], srv->round_ev[r], 0);
                        if (e != cudaSuccess) {
                            run_status = GATEAU_ECUDA;
                            run_error = std::string("round launch: ") + cudaGetErrorString(e);
                        }
                        for (size_t m = 0; m < members.size() && run_status == GATEAU_OK; ++m) {
                            Req& q = R[members[m]];
                            post_chunk(q, static_cast<int>(q.launched % depth), nts[m]);
                        }
                    }
                }
                if (run_status != GATEAU_OK) break;
                if (enqueued) {
                    for (size_t m = 0; m < members.size(); ++m) {
                        Req& q = R[members[m]];
                        Slot& sl = q.slot[q.launched % depth];
                        sl.busy = true;
                        sl.t0 = q.next_t0;
                        sl.nt = nts[m];
                        if (dry) sl.t_end = round_end[r];
                        q.next_t0 += nts[m];
                        ++q.launched;
                    }
                    ++rounds_launched;
                    round_members += static_cast<long long>(members.size());
                    count_overlap();
                    progress = true;
                }
            }
        } else {
            for (int i = 0; i < n && run_status == GATEAU_OK; ++i) {
                Req& q = R[i];
                if (q.state != kActive) continue;
                while (q.launched - q.retired < depth && q.next_t0 < q.r.nt) {
                    Slot& sl = q.slot[q.launched % depth];
                    const long long len = std::min(q.chunk, q.r.nt - q.next_t0);
                    if (dry) {
                        const double work = static_cast<double>(len) * q.r.n_pix * q.r.n_ch * d.dry_seconds_per_sample;
                        const double start = std::max(now(), stream_free[q.stream]);
                        sl.t_end = start + work;
                        stream_free[q.stream] = sl.t_end;
                    } else {
                        cudaStream_t st = srv->streams[q.stream];
                        gateau_status gs = gateau_run(q.plan, q.next_t0, len, sl.d_out, st);
                        if (gs != GATEAU_OK) {                 // nothing of this chunk was enqueued
                            cudaStreamSynchronize(st);         // earlier chunks of this request
                            finish(q, i, kFailed);
                            progress = true;
                            break;
                        }
                        if (!post_chunk(q, static_cast<int>(q.launched % depth), len)) break;
                    }
                    sl.busy = true;
                    sl.t0 = q.next_t0;
                    sl.nt = len;
                    q.next_t0 += len;
                    ++q.launched;
                    progress = true;
                    count_overlap();
                }
            }
        }
        if (run_status != GATEAU_OK) break;

        // 4. nothing to do: wait for the next event (a chunk, or an arrival)
        if (!progress) {
            bool busy = false;
            double t_next = 1e300;                 // dry run: the next virtual event
            for (const Req& q : R)
                if (q.state == kActive && q.retired < q.launched) {
                    busy = true;
                    t_next = std::min(t_next, q.slot[q.retired % depth].t_end);
                }
            const double t_now = now();
            const bool arrival_ahead = next < n && R[next].state == kPending && requests[next].arrival_s > t_now;
            if (arrival_ahead) t_next = std::min(t_next, requests[next].arrival_s);
            // Nothing in flight, no plan being built and no arrival still to come: the pending
            // requests cannot be admitted (cannot happen with the admission rules above; kept as a
            // guard against spinning).
            if (!busy && n_building == 0 && !arrival_ahead) break;
            if (n_building > 0) busy = true;
            if (dry) {
                vclock = std::max(vclock, t_next);
            } else {
                const double wait = busy ? 20e-6 : std::min(1e-3, std::max(0.0, t_next - t_now));
                std::this_thread::sleep_for(std::chrono::duration<double>(wait));
            }
        }
    }

    if (use_builders) {                            // no build left in flight
        {
            std::lock_guard<std::mutex> lk(B.mu);
            B.stop = true;
            B.todo.clear();
        }
        B.cv.notify_all();
        for (std::thread& th : B.threads) th.join();
        for (auto& pr : B.done)
            if (pr.second) release(user, pr.first, pr.second);
        for (auto& pr : failed_builds) release(user, pr.first, pr.second);
        for (Req& q : R)
            if (q.state == kBuilding) q.state = kFailed;
    }
    if (run_status != GATEAU_OK) {                 // release whatever is still admitted
        if (srv->batch_stream) cudaStreamSynchronize(srv->batch_stream);
        for (cudaStream_t st : srv->streams) cudaStreamSynchronize(st);
        for (int i = 0; i < n; ++i)
            if (R[i].state == kActive) finish(R[i], i, kFailed);
    }

    if (stats) {
        gateau_server_stats st{};
        st.n_requests = n;
        std::vector<double> lat;
        double samples = 0.0, last = 0.0;
        for (const Req& q : R) {
            if (q.state == kDone) {
                ++st.n_done;
                lat.push_back(q.t_done - q.r.arrival_s);
                samples += static_cast<double>(q.r.nt) * q.r.n_pix * q.r.n_ch;
                last = std::max(last, q.t_done);
            } else if (q.state == kFailed) {
                ++st.n_failed;
            }
        }
        st.p50_latency_s = percentile(lat, 0.50);
        st.p99_latency_s = percentile(lat, 0.99);
        double sum = 0.0, mx = 0.0;
        for (double v : lat) {
            sum += v;
            mx = std::max(mx, v);
        }
        st.mean_latency_s = lat.empty() ? 0.0 : sum / lat.size();
        st.max_latency_s = mx;
        st.makespan_s = last;
        st.detector_samples = samples;
        st.throughput = last > 0.0 ? samples / last : 0.0;
        st.peak_bytes = peak_bytes;
        st.peak_active = peak_active;
        st.overlap = overlap_n ? overlap_sum / overlap_n : 0.0;
        st.rounds = rounds_launched;
        st.mean_round = rounds_launched ? static_cast<double>(round_members) / rounds_launched : 0.0;
        *stats = st;
    }
    if (run_status != GATEAU_OK) return server_fail(run_status, run_error);
    return GATEAU_OK;
}

gateau_status gateau_server_request_result(gateau_server* srv, int request, int* state, double* latency_s,
                                           double* admitted_s, double* checksum2) {
    if (!srv) return server_fail(GATEAU_EINVAL, "server is NULL");
    if (request < 0 || request >= static_cast<int>(srv->reqs.size()))
        return server_fail(GATEAU_EINVAL, "request index out of range of the last run");
    const Req& q = srv->reqs[request];
    if (state) *state = q.state;
    if (latency_s) *latency_s = q.state == kDone ? q.t_done - q.r.arrival_s : 0.0;
    if (admitted_s) *admitted_s = q.t_admit;
    if (checksum2) {
        checksum2[0] = q.sum;
        checksum2[1] = q.sumsq;
    }
    return GATEAU_OK;
}

}  // extern "C"
