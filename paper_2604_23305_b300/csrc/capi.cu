// C ABI of the simulator: plan object, setters, run orchestration.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "gateau_internal.h"

using namespace gateau;

namespace {

thread_local std::string g_last_error;

gateau_status fail(gateau_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define GATEAU_CUDA(call)                                                                         \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(e_ == cudaErrorMemoryAllocation ? GATEAU_ENOMEM : GATEAU_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                       \
    } while (0)

// Grow-only device buffer in the stream-ordered allocator.  Allocation and release run on the
// owning plan's memory stream, which first waits for the work the plan enqueued, so freeing a
// plan's memory never synchronises the device (a server destroys finished requests' plans while
// others run).
struct MemOrder {
    cudaStream_t mem = nullptr;        // allocation / release stream (non-blocking)
    cudaStream_t after[2] = {nullptr, nullptr};   // streams whose enqueued work must finish first
    bool after_used[2] = {false, false};
    cudaError_t ready() {
        if (mem) return cudaSuccess;
        static std::once_flag pool_once;
        std::call_once(pool_once, [] {
            // Keep freed blocks in this process's default pool instead of returning them to the
            // driver at every synchronisation (a process-local setting of the pool).
            int dev = 0;
            cudaMemPool_t pool;
            if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                unsigned long long keep = ~0ull;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            }
        });
        return cudaStreamCreateWithFlags(&mem, cudaStreamNonBlocking);
    }
    // Order the memory stream after everything enqueued so far on the plan's run streams.
    cudaError_t fence() {
        for (int i = 0; i < 2; ++i) {
            if (!after_used[i]) continue;
            cudaEvent_t e = nullptr;
            cudaError_t err = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
            if (err != cudaSuccess) return err;
            err = cudaEventRecord(e, after[i]);
            if (err == cudaSuccess) err = cudaStreamWaitEvent(mem, e, 0);
            cudaEventDestroy(e);                      // released once the wait is resolved
            if (err != cudaSuccess) return err;
        }
        return cudaSuccess;
    }
};

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t n, MemOrder& mo) {
        if (n <= bytes) return cudaSuccess;
        cudaError_t e = mo.ready();
        if (e != cudaSuccess) return e;
        release(mo);
        e = cudaMallocAsync(&p, n, mo.mem);
        if (e == cudaSuccess) e = cudaStreamSynchronize(mo.mem);   // usable on any stream from here
        if (e == cudaSuccess) {
            bytes = n;
        } else {
            p = nullptr;
        }
        return e;
    }
    void release(MemOrder& mo) {
        if (p && mo.ready() == cudaSuccess && mo.fence() == cudaSuccess) cudaFreeAsync(p, mo.mem);
        p = nullptr;
        bytes = 0;
    }
    template <class T>
    T* as() const {
        return static_cast<T*>(p);
    }
};

}  // namespace

namespace {
// Tile autotuner cache: shape class -> (channel groups, B-ring depth), shared by every plan of the
// process.  The class is the channel count in 16-channel blocks, which fixes every candidate's
// group width and ring depths; spaxels and spectral points change how many items and stages a
// launch has, not which tiles fit.
std::mutex g_tune_mu;
std::map<int, std::pair<int, int>> g_tune_cache;
}  // namespace

namespace gateau {
// Lets other translation units report through gateau_last_error().
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace gateau

struct gateau_plan {
    gateau_plan_desc desc{};
    std::vector<double> pix_off;      // [n_pix][2]
    std::vector<double> nu, w;
    int Kp = 0;

    // setters' state
    bool has_cube = false, has_screen = false, has_table = false, has_cascade = false, has_disp = false,
         has_scan = false, has_pink = false;
    int n_az = 0, n_el = 0;
    double az0 = 0, daz = 0, el0 = 0, del = 0;
    int nx = 0, ny = 0;
    double pitch = 0;
    int n_pwv = 0;
    double pwv_min = 0, dpwv = 0;
    std::vector<float> table_raw;     // the table [n_pwv][n_freq] as last set (values before any conversion)
    bool table_is_opacity = false;    // table_raw holds opacities (else transmissions, tau = -ln t)
    double screen_mean = 0;           // mean PWV of the screen (mm)
    std::vector<StageSpec> stages;
    int disp_kind = 0, n_ch = 0;
    std::vector<double> eta_filt;      // [n_ch][n_freq]
    std::vector<double> pink_A, pink_alpha;
    bool pink_auto = false;          // pink level from the reference spectrum's NEP^2 (knee at 1 Hz)
    int scan_kind = GATEAU_SCAN_STARE;
    double sp[kMaxScanParams] = {0};
    double phi0 = 0, theta0 = 0;
    long long n_custom = 0;

    // brightness-temperature output (gateau_set_output_kelvin)
    bool kelvin = false;
    double dip_lo = 0, dip_hi = 0;
    int dip_n = 0;
    std::vector<double> tb_a, tb_b;  // the skydip fit, read back from the device
    long long tk_n = 0;              // > 0: exact (Timmer-Koenig) pink noise over samples [0, tk_n)

    // derived host tables
    std::vector<double> c0, c1, c2;
    int n_pole = 0;
    std::vector<double> pink_a, pink_r, pink_d;
    bool dirty = true;
    bool ref_dirty = true;           // the reference spectrum (screen mean, table, theta0, cascade) changed
    int tile_groups = 0;             // fused tiles: channel groups (0: the default rule), set or tuned
    int tile_ring_b = 0;             // fused tiles: deepest B ring (0: the default)
    double tune_ms = 0.0;            // the tuned configuration's time on the tuning sample (0: not measured)

    // device memory
    DevBuf d_pix, d_cube, d_cube_raw, d_screen, d_tau, d_tau_rows, d_custom, d_c, d_HGQ, d_fusedB, d_pink, d_state, d_status;
    DevBuf d_tb, d_dip;              // skydip fit [2][n_ch] float for the epilogues; FP64 scratch of the fit
    DevBuf d_tk, d_tkz;              // Timmer-Koenig pink TOD [tk_n][n_pix][n_ch]; its FFT scratch
    DevBuf d_hw, d_cm;               // common-mode reduction: eta_filt w (FP64); log eta_z, S_j, PWV sum
    DevBuf d_ref;                    // per channel: k_B 1e9 S_ref and N_ref of the reference spectrum
    DevBuf d_tune;                   // tile autotuner: output of the timed sample runs
    bool cube_scale_dirty = true;    // d_cube = d_cube_raw * c2 / k_B must be recomputed
    DevBuf d_rows, d_tiles, d_X, d_agg, d_stage[2];
    FusedOperands fused{};
    TensorMapBytes tm_tau{}, tm_tau_s{}, tm_cube{}, tm_cube_s{};
    bool maps_dirty = true;
    int n_ch_pad = 0;
    int n_sm = 148;
    long long next_t0 = 0;
    cudaStream_t last_stream = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_done[2] = {nullptr, nullptr}, ev_copied[2] = {nullptr, nullptr};
    // phase timing: pairs of events per phase and run, resolved in gateau_plan_get_timing
    bool timing = false;
    struct TimedRun { cudaEvent_t ev[GATEAU_PHASE_COUNT][2]; bool used[GATEAU_PHASE_COUNT]; };
    std::vector<TimedRun> timed;
    std::vector<cudaEvent_t> ev_pool;
    long long runs = 0, launches = 0;

    MemOrder mo;                     // stream order of this plan's device allocations
    bool ran = false;                // a run was enqueued (on last_stream)

    // Point the memory order at the streams this plan enqueued work on.
    void track_streams() {
        mo.after[0] = last_stream;
        mo.after_used[0] = ran;
        mo.after[1] = copy_stream;
        mo.after_used[1] = copy_stream != nullptr;
    }

    ~gateau_plan() {
        track_streams();
        DevBuf* bufs[] = {&d_pix, &d_cube, &d_cube_raw, &d_screen, &d_tau, &d_tau_rows, &d_custom, &d_c, &d_HGQ, &d_fusedB, &d_pink,
                          &d_state, &d_status, &d_rows, &d_tiles, &d_X, &d_agg, &d_stage[0], &d_stage[1],
                          &d_tb, &d_dip, &d_tk, &d_tkz, &d_hw, &d_cm, &d_ref, &d_tune};
        for (DevBuf* b : bufs) b->release(mo);
        if (mo.mem) cudaStreamDestroy(mo.mem);       // its pending frees still complete
        for (int i = 0; i < 2; ++i) {
            if (ev_done[i]) cudaEventDestroy(ev_done[i]);
            if (ev_copied[i]) cudaEventDestroy(ev_copied[i]);
        }
        if (copy_stream) cudaStreamDestroy(copy_stream);
        for (TimedRun& t : timed)
            for (int ph = 0; ph < GATEAU_PHASE_COUNT; ++ph)
                if (t.used[ph]) {
                    cudaEventDestroy(t.ev[ph][0]);
                    cudaEventDestroy(t.ev[ph][1]);
                }
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    }
};

namespace {

// Grow a plan buffer; the old contents are released after the plan's enqueued work.
cudaError_t grow(gateau_plan* p, DevBuf& b, size_t n) {
    p->track_streams();
    return b.ensure(n, p->mo);
}

size_t device_bytes(const gateau_plan* p) {
    const DevBuf* bufs[] = {&p->d_pix, &p->d_cube, &p->d_cube_raw, &p->d_screen, &p->d_tau, &p->d_tau_rows, &p->d_custom, &p->d_c,
                            &p->d_HGQ, &p->d_fusedB, &p->d_pink, &p->d_state, &p->d_status, &p->d_rows,
                            &p->d_tiles, &p->d_X, &p->d_agg, &p->d_stage[0], &p->d_stage[1], &p->d_tb, &p->d_dip,
                            &p->d_tk, &p->d_tkz, &p->d_hw, &p->d_cm, &p->d_ref, &p->d_tune};
    size_t s = 0;
    for (const DevBuf* b : bufs) s += b->bytes;
    return s;
}

cudaMemcpyKind kind_of(int mem) { return mem == GATEAU_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }

gateau_status check_mem(int mem) {
    if (mem != GATEAU_MEM_HOST && mem != GATEAU_MEM_DEVICE) return fail(GATEAU_EINVAL, "mem must be GATEAU_MEM_HOST or GATEAU_MEM_DEVICE");
    return GATEAU_OK;
}

// Copy a device or host float array to host memory.
gateau_status fetch_floats(const float* src, size_t n, int mem, std::vector<float>& out) {
    out.resize(n);
    if (mem == GATEAU_MEM_DEVICE) {
        GATEAU_CUDA(cudaMemcpy(out.data(), src, n * sizeof(float), cudaMemcpyDeviceToHost));
    } else {
        memcpy(out.data(), src, n * sizeof(float));
    }
    return GATEAU_OK;
}

// Contraction operands in device units (w in GHz, X in kelvin), FP64 per (channel, point):
//   H = eta w_GHz;  G = H gamma (nu_GHz + beta);  Q = eta^2 w_GHz
// with gamma = h 1e9 / k_B and beta = 2 Delta_Al / (eta_pb h 1e9) (Sect. 2.5 Eq. 16, Sect. 2.6 Eq. 17),
// formed per element where they are used (the reference integrals, the FP32 operands, the split-BF16
// tiles) rather than stored as three [n_ch][Kp] FP64 matrices.
FilterOperands filter_operands(const gateau_plan* p) {
    const gateau_plan_desc& d = p->desc;
    FilterOperands f;
    f.eta = p->eta_filt.data();
    f.w = p->w.data();
    f.nu = p->nu.data();
    f.nf = d.n_freq;
    f.gamma = kH * 1e9 / kKB;
    f.beta = 2.0 * d.delta_al_J / (d.eta_pb * kH * 1e9);
    return f;
}

// Transmission of the reference sky per point: exp(-csc(theta_0) tau_z) at the screen's mean PWV,
// Zenith opacity of table entry i in FP64: the value itself, or -ln t of a transmission t (floored
// at 1e-30, so that a zero transmission stays finite).
static double table_opacity(const gateau_plan* p, size_t i) {
    const double v = p->table_raw[i];
    return p->table_is_opacity ? v : -log(std::max(v, 1e-30));
}

// tau_z interpolated linearly between the table's PWV rows (clamped to the table), Eq. 10 at the
// scan's base elevation.  1 before the table is set.
std::vector<double> reference_transmission(const gateau_plan* p) {
    const int nf = p->desc.n_freq;
    std::vector<double> eref(nf, 1.0);
    if (p->table_raw.empty() || p->n_pwv < 2) return eref;
    double u = (p->screen_mean - p->pwv_min) / p->dpwv;
    u = std::min(std::max(u, 0.0), static_cast<double>(p->n_pwv - 1));
    const int j = std::min(static_cast<int>(floor(u)), p->n_pwv - 2);
    const double f = u - j;
    const double sn = sin(p->theta0);
    const double csc = sn > 1e-3 ? 1.0 / sn : 1.0;      // elevations below 0.06 deg: a zenith reference
    for (int k = 0; k < nf; ++k) {
        const double tau = (1.0 - f) * table_opacity(p, static_cast<size_t>(j) * nf + k) +
                           f * table_opacity(p, static_cast<size_t>(j + 1) * nf + k);
        eref[k] = exp(-csc * tau);
    }
    return eref;
}

// Reference spectrum: the source-free collapse (Sect. 2.5) at the screen's mean PWV and the
// base elevation theta_0 (Eq. 10), X_ref = c0 + c1 (1 - e_ref).  Both contraction paths run on
// D = X - X_ref instead of X.  D stays small wherever the line of sight sees about the mean sky,
// so the FP32 and split-BF16 rounding is relative to the sky's fluctuation rather than to the
// whole loading, and the source term, orders of magnitude below the atmosphere's, survives it.
// The integrals of Eqs. 16-17 are linear in X plus a term in X^2, so with X = D + X_ref
//   sum H X           = sum H D + S_ref,                         S_ref = sum H X_ref
//   sum G X + Q X^2   = sum (G + 2 Q X_ref) D + Q D^2 + N_ref,   N_ref = sum G X_ref + Q X_ref^2:
// only the G operand changes, and the epilogues add two per-channel constants.  The kernels form
// D = c_ref - c1 e + e P'_src with c_ref = fp32(c1 e_ref); X_ref is taken as
// (c0 + c1) / k_B - c_ref in FP64, so X = D + X_ref holds for the values the kernels use.
gateau_status build_reference(gateau_plan* p) {
    const gateau_plan_desc& d = p->desc;
    const int nf = d.n_freq, Kp = p->Kp, n_ch = p->n_ch;
    const std::vector<double> eref = reference_transmission(p);
    std::vector<float> c1f(Kp, 0.f), cref(Kp, 0.f);
    std::vector<double> xref(Kp, 0.0);
    for (int k = 0; k < nf; ++k) {
        c1f[k] = static_cast<float>(p->c1[k] / kKB);
        cref[k] = static_cast<float>(p->c1[k] / kKB * eref[k]);
        xref[k] = (p->c0[k] + p->c1[k]) / kKB - static_cast<double>(cref[k]);
    }
    // c_ref [Kp], then per 16-point stage for the fused kernel: [Kp/16][c_ref, c1][16]
    std::vector<float> cv(cref);
    const int ks = fused_kstage();
    for (int b = 0; b < Kp / ks; ++b) {
        for (int k = 0; k < ks; ++k) cv.push_back(cref[b * ks + k]);
        for (int k = 0; k < ks; ++k) cv.push_back(c1f[b * ks + k]);
    }
    GATEAU_CUDA(cudaMemcpy(p->d_c.as<float>() + 3 * static_cast<size_t>(Kp), cv.data(), cv.size() * sizeof(float),
                           cudaMemcpyHostToDevice));

    FilterOperands fo = filter_operands(p);
    fo.xref = xref.data();
    const int stride = p->n_ch_pad;
    std::vector<float> rv(2 * static_cast<size_t>(stride), 0.f);
    for (int c = 0; c < n_ch; ++c) {
        double s_ref = 0.0, n_ref = 0.0;
        for (int k = 0; k < nf; ++k) {
            double h, g, q;
            fo.at(c, k, h, g, q);
            s_ref += h * xref[k];
            n_ref += (g + q * xref[k]) * xref[k];
        }
        rv[c] = static_cast<float>(kKB * 1e9 * s_ref);     // P_KID of the reference (W)
        rv[stride + c] = static_cast<float>(n_ref);
    }
    GATEAU_CUDA(grow(p, p->d_ref, rv.size() * sizeof(float)));
    GATEAU_CUDA(cudaMemcpy(p->d_ref.p, rv.data(), rv.size() * sizeof(float), cudaMemcpyHostToDevice));

    if (d.precision == GATEAU_PREC_FP32) {
        std::vector<float> hgq(3 * static_cast<size_t>(p->n_ch_pad) * Kp, 0.f);
        const size_t mat = static_cast<size_t>(p->n_ch_pad) * Kp;
        for (int c = 0; c < n_ch; ++c)
            for (int k = 0; k < nf; ++k) {
                double h, g, q;
                fo.at(c, k, h, g, q);
                const size_t i = static_cast<size_t>(c) * Kp + k;
                hgq[i] = static_cast<float>(h);
                hgq[mat + i] = static_cast<float>(fo.gprime(g, q, k));
                hgq[2 * mat + i] = static_cast<float>(q);
            }
        GATEAU_CUDA(grow(p, p->d_HGQ, hgq.size() * sizeof(float)));
        GATEAU_CUDA(cudaMemcpy(p->d_HGQ.p, hgq.data(), hgq.size() * sizeof(float), cudaMemcpyHostToDevice));
    } else {
        // channel groups of at most 176 (the accumulators of a group fill 352 of the 512 TMEM
        // columns): the default is the fewest groups; a set or tuned count may use more
        const int n_groups = p->tile_groups > 0 ? p->tile_groups : (n_ch + 175) / 176;
        p->fused.n_groups = n_groups;
        p->fused.n_half = ((n_ch + n_groups - 1) / n_groups + 15) / 16 * 16;
        p->fused.n_kstage = Kp / fused_kstage();
        p->fused.ring_b = p->tile_ring_b > 0 ? p->tile_ring_b : kDefaultRingB;
        std::vector<uint16_t> tiled;
        size_t stage_elems = 0;
        fused_tile_operands(fo, n_ch, Kp, p->fused.n_half, p->fused.n_groups, tiled, stage_elems);
        GATEAU_CUDA(grow(p, p->d_fusedB, tiled.size() * sizeof(uint16_t)));
        GATEAU_CUDA(cudaMemcpy(p->d_fusedB.p, tiled.data(), tiled.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
        p->fused.B = p->d_fusedB.as<uint16_t>();
        p->fused.stage_elems = stage_elems;
    }
    p->ref_dirty = false;
    return GATEAU_OK;
}

// Rebuild the derived tables (cascade collapse, channel grouping, skydip, pink filters) and upload them.
gateau_status finalize_tables(gateau_plan* p) {
    const gateau_plan_desc& d = p->desc;
    const int nf = d.n_freq, Kp = p->Kp;
    // cascade collapse (Sect. 2.5)
    std::vector<PrimStage> prim;
    std::string err;
    if (!expand_stages(p->stages, p->nu, prim, err)) return fail(GATEAU_EINVAL, "%s", err.c_str());
    collapse_cascade(p->nu, prim, d.T_atm_K, d.T_cmb_K, d.eta_taper, d.rho_surf_m, d.eta_pol, p->c0, p->c1, p->c2);
    // per-frequency device vectors (kelvin units: divide by k_B): c0, c1, c2; then c_ref and its
    // per-stage tiling, written by build_reference
    std::vector<float> cv(3 * static_cast<size_t>(Kp), 0.f);
    for (int k = 0; k < nf; ++k) {
        cv[k] = static_cast<float>(p->c0[k] / kKB);
        cv[Kp + k] = static_cast<float>(p->c1[k] / kKB);
        cv[2 * Kp + k] = static_cast<float>(p->c2[k] / kKB);
    }
    GATEAU_CUDA(grow(p, p->d_c, 6 * static_cast<size_t>(Kp) * sizeof(float)));
    GATEAU_CUDA(cudaMemcpy(p->d_c.p, cv.data(), cv.size() * sizeof(float), cudaMemcpyHostToDevice));
    p->fused.c_tiled = p->d_c.as<float>() + 4 * static_cast<size_t>(Kp);
    p->cube_scale_dirty = true;

    const int n_ch = p->n_ch;
    p->n_ch_pad = (n_ch + 63) / 64 * 64;

    // brightness-temperature scale (Sect. 2.7): the skydip runs on the device (FP64), its fit
    // comes back for gateau_plan_get_vector and for the pink coefficients below
    if (p->kelvin) {
        const size_t hw_n = static_cast<size_t>(n_ch) * nf;
        std::vector<double> dip(hw_n + 2 * static_cast<size_t>(nf) + 2 * static_cast<size_t>(n_ch), 0.0);
        for (int c = 0; c < n_ch; ++c)
            for (int k = 0; k < nf; ++k) dip[static_cast<size_t>(c) * nf + k] = p->eta_filt[static_cast<size_t>(c) * nf + k] * p->w[k];
        for (int k = 0; k < nf; ++k) {
            dip[hw_n + k] = p->c0[k];
            dip[hw_n + nf + k] = p->c1[k];
        }
        GATEAU_CUDA(grow(p, p->d_dip, dip.size() * sizeof(double)));
        const size_t tb_stride = (static_cast<size_t>(n_ch) + 15) / 16 * 16;
        GATEAU_CUDA(grow(p, p->d_tb, 2 * tb_stride * sizeof(float)));
        GATEAU_CUDA(cudaMemset(p->d_tb.p, 0, 2 * tb_stride * sizeof(float)));
        GATEAU_CUDA(cudaMemcpy(p->d_dip.p, dip.data(), (hw_n + 2 * static_cast<size_t>(nf)) * sizeof(double),
                               cudaMemcpyHostToDevice));
        double* ab = p->d_dip.as<double>() + hw_n + 2 * static_cast<size_t>(nf);
        GATEAU_CUDA(launch_skydip_fit(p->d_dip.as<double>(), p->d_dip.as<double>() + hw_n, p->d_tau.as<float>(), nf, Kp,
                                      p->n_pwv, p->pwv_min, p->dpwv, 1.0 / sin(p->theta0), d.T_atm_K, p->dip_lo,
                                      p->dip_hi, p->dip_n, n_ch, ab, p->d_tb.as<float>(), static_cast<int>(tb_stride),
                                      nullptr));
        std::vector<double> abh(2 * static_cast<size_t>(n_ch));
        GATEAU_CUDA(cudaMemcpy(abh.data(), ab, abh.size() * sizeof(double), cudaMemcpyDeviceToHost));
        p->tb_a.assign(abh.begin(), abh.begin() + n_ch);
        p->tb_b.assign(abh.begin() + n_ch, abh.end());
        p->d_dip.release(p->mo);
    } else {
        p->tb_a.clear();
        p->tb_b.clear();
    }

    // pink level with no A given: the knee at 1 Hz, A = NEP^2 (Eq. 17) of the source-free sky at the
    // screen's mean PWV and the base elevation, the one-sided white PSD of Eq. 18
    if (p->pink_auto) {
        const std::vector<double> eref = reference_transmission(p);
        const double gr = 2.0 * d.delta_al_J / d.eta_pb;
        p->pink_A.assign(n_ch, 0.0);
        for (int c = 0; c < n_ch; ++c) {
            double shot = 0.0, bunching = 0.0, absorbed = 0.0;
            for (int k = 0; k < nf; ++k) {
                const double P = p->c0[k] + p->c1[k] * (1.0 - eref[k]);
                const double ew = p->eta_filt[static_cast<size_t>(c) * nf + k] * p->w[k];
                shot += ew * P * kH * p->nu[k];
                bunching += ew * p->eta_filt[static_cast<size_t>(c) * nf + k] * P * P;
                absorbed += ew * P;
            }
            p->pink_A[c] = 2.0 * (shot + bunching + gr * absorbed);
        }
    }

    // pink filters (Sect. 2.6, Eq. 20)
    p->n_pole = pink_pole_count(d.pink_f_min_hz, d.f_sample_hz);
    const int np = p->n_pole;
    p->pink_a.assign(static_cast<size_t>(n_ch) * np, 0.0);
    p->pink_r.assign(static_cast<size_t>(n_ch) * np, 0.0);
    p->pink_d.assign(n_ch, 0.0);
    for (int c = 0; c < n_ch; ++c) {
        const double A = p->has_pink ? p->pink_A[c] : 0.0;
        const double al = p->has_pink ? p->pink_alpha[c] : 1.0;
        pink_design_channel(al, A, d.pink_f_min_hz, d.f_sample_hz, np, &p->pink_a[static_cast<size_t>(c) * np],
                            &p->pink_r[static_cast<size_t>(c) * np], &p->pink_d[c]);
    }
    std::vector<float> pk(static_cast<size_t>(n_ch) * (2 * np + 1));
    // kelvin output: the pink term enters as tb_a P_pn, i.e. residues and direct term times tb_a
    // (the filter states do not depend on them)
    for (size_t i = 0; i < p->pink_a.size(); ++i) {
        const double sc = p->kelvin ? p->tb_a[i / np] : 1.0;
        pk[i] = static_cast<float>(p->pink_a[i]);
        pk[p->pink_a.size() + i] = static_cast<float>(sc * p->pink_r[i]);
    }
    for (int c = 0; c < n_ch; ++c)
        pk[2 * p->pink_a.size() + c] = static_cast<float>((p->kelvin ? p->tb_a[c] : 1.0) * p->pink_d[c]);
    GATEAU_CUDA(grow(p, p->d_pink, pk.size() * sizeof(float)));
    GATEAU_CUDA(cudaMemcpy(p->d_pink.p, pk.data(), pk.size() * sizeof(float), cudaMemcpyHostToDevice));
    // exact pink noise (Sect. 2.6, Timmer & Koenig): the whole scan's realisation, once per plan
    if (p->tk_n > 0 && (d.noise_flags & GATEAU_NOISE_PINK)) {
        const long long M = tk_length(p->tk_n);
        const size_t n_pairs = static_cast<size_t>(d.n_pix) * ((n_ch + 1) / 2);
        const size_t zbytes = n_pairs * static_cast<size_t>(M) * sizeof(float2);
        GATEAU_CUDA(grow(p, p->d_tk, static_cast<size_t>(p->tk_n) * d.n_pix * n_ch * sizeof(float)));
        GATEAU_CUDA(grow(p, p->d_tkz, 2 * zbytes + 2 * static_cast<size_t>(n_ch) * sizeof(double)));
        std::vector<double> par(2 * static_cast<size_t>(n_ch), 0.0);
        for (int c = 0; c < n_ch; ++c) {
            par[c] = p->has_pink ? p->pink_A[c] : 0.0;
            par[n_ch + c] = p->has_pink ? p->pink_alpha[c] : 1.0;
        }
        uint8_t* zb = p->d_tkz.as<uint8_t>();
        double* dpar = reinterpret_cast<double*>(zb + 2 * zbytes);
        GATEAU_CUDA(cudaMemcpy(dpar, par.data(), par.size() * sizeof(double), cudaMemcpyHostToDevice));
        GATEAU_CUDA(launch_tk_realise(dpar, dpar + n_ch, d.f_sample_hz, static_cast<uint32_t>(d.seed & 0xffffffffull),
                                      static_cast<uint32_t>(d.seed >> 32), d.n_pix, n_ch, p->tk_n,
                                      p->kelvin ? p->d_tb.as<float>() : nullptr, reinterpret_cast<float2*>(zb),
                                      reinterpret_cast<float2*>(zb + zbytes), p->d_tk.as<float>(), nullptr));
        GATEAU_CUDA(cudaStreamSynchronize(nullptr));
        p->d_tkz.release(p->mo);
    }
    const size_t state_bytes = static_cast<size_t>(d.n_pix) * n_ch * np * sizeof(float);
    if (p->d_state.bytes < state_bytes) {
        GATEAU_CUDA(grow(p, p->d_state, state_bytes));
        GATEAU_CUDA(cudaMemset(p->d_state.p, 0, state_bytes));
    }
    p->dirty = false;
    p->ref_dirty = true;
    return GATEAU_OK;
}

gateau_status finalize(gateau_plan* p) {
    if (p->dirty) {
        const gateau_status st = finalize_tables(p);
        if (st != GATEAU_OK) return st;
    }
    return p->ref_dirty ? build_reference(p) : GATEAU_OK;
}

DevTables make_tables(const gateau_plan* p) {
    const gateau_plan_desc& d = p->desc;
    DevTables T{};
    T.n_pix = d.n_pix;
    T.pix_off = p->d_pix.as<double>();
    T.pix_trig = T.pix_off ? T.pix_off + 2 * static_cast<size_t>(d.n_pix) : nullptr;
    T.pix_trig_f = T.pix_off ? reinterpret_cast<const float*>(T.pix_off + 6 * static_cast<size_t>(d.n_pix)) : nullptr;
    T.f_sample = d.f_sample_hz;
    T.h_column = d.h_column_m;
    T.wind = d.wind_mps;
    T.scan_kind = p->scan_kind;
    for (int i = 0; i < kMaxScanParams; ++i) T.sp[i] = p->sp[i];
    T.phi0 = p->phi0;
    T.theta0 = p->theta0;
    T.custom = p->d_custom.as<double>();
    T.n_custom = p->n_custom;
    T.screen = p->d_screen.as<float>();
    T.nx = p->nx;
    T.ny = p->ny;
    T.pitch = p->pitch;
    T.tau = p->d_tau.as<float>();
    T.n_pwv = p->n_pwv;
    T.pwv_min = p->pwv_min;
    T.dpwv = p->dpwv;
    T.cube = p->d_cube.as<float>();
    T.n_az = p->n_az;
    T.n_el = p->n_el;
    T.az0 = p->az0;
    T.daz = p->daz;
    T.el0 = p->el0;
    T.del = p->del;
    T.n_freq = d.n_freq;
    T.Kp = p->Kp;
    T.c0 = p->d_c.as<float>();
    T.c1 = T.c0 + p->Kp;
    T.c2 = T.c0 + 2 * p->Kp;
    T.cref = T.c0 + 3 * p->Kp;
    T.ref_pk = p->d_ref.as<float>();
    T.ref_n = T.ref_pk ? T.ref_pk + p->n_ch_pad : nullptr;
    T.n_ch = p->n_ch;
    T.n_ch_pad = p->n_ch_pad;
    const size_t mat = static_cast<size_t>(p->n_ch_pad) * p->Kp;
    T.H = p->d_HGQ.as<float>();
    T.G = T.H ? T.H + mat : nullptr;
    T.Q = T.H ? T.H + 2 * mat : nullptr;
    T.kb1e9 = static_cast<float>(kKB * 1e9);
    T.kB = static_cast<float>(kKB);
    T.noise_scale = static_cast<float>(1e9 * d.f_sample_hz);
    T.key0 = static_cast<uint32_t>(d.seed & 0xffffffffull);
    T.key1 = static_cast<uint32_t>(d.seed >> 32);
    T.noise_flags = d.noise_flags;
    T.n_pole = p->n_pole;
    const size_t pa = static_cast<size_t>(p->n_ch) * p->n_pole;
    T.pink_a = p->d_pink.as<float>();
    T.pink_r = T.pink_a + pa;
    T.pink_d = T.pink_a + 2 * pa;
    T.tb_a = p->kelvin ? p->d_tb.as<float>() : nullptr;
    T.tb_b = p->kelvin ? T.tb_a + (p->n_ch + 15) / 16 * 16 : nullptr;
    T.status = p->d_status.as<unsigned int>();
    return T;
}

gateau_status check_complete(const gateau_plan* p) {
    if (!p->has_cube) return fail(GATEAU_ESTATE, "source cube not set (gateau_set_source_cube)");
    if (!p->has_screen) return fail(GATEAU_ESTATE, "atmosphere screen not set (gateau_set_atmosphere_screen)");
    if (!p->has_table) return fail(GATEAU_ESTATE, "atmosphere table not set (gateau_set_atmosphere_table)");
    if (!p->has_cascade) return fail(GATEAU_ESTATE, "cascade not set (gateau_set_cascade)");
    if (!p->has_disp) return fail(GATEAU_ESTATE, "dispersive element not set (gateau_set_dispersive_element)");
    if (!p->has_scan) return fail(GATEAU_ESTATE, "scan not set (gateau_set_scan)");
    return GATEAU_OK;
}

gateau_status validate_run(const gateau_plan* p, long long t0, long long nt, const void* out) {
    gateau_status st = check_complete(p);
    if (st != GATEAU_OK) return st;
    if (t0 < 0 || nt <= 0) return fail(GATEAU_EINVAL, "need t0 >= 0 and nt > 0 (got t0=%lld nt=%lld)", t0, nt);
    if (nt > (1LL << 31) / p->desc.n_pix)       // nt * n_pix > 2^31, compared without forming the product
        return fail(GATEAU_EINVAL, "nt * n_pix must stay below 2^31 rows per call");
    if (t0 > (1LL << 62)) return fail(GATEAU_EINVAL, "t0 must stay below 2^62");   // t0 + nt cannot overflow
    if (!out) return fail(GATEAU_EINVAL, "out is NULL");
    if ((p->desc.noise_flags & GATEAU_NOISE_PINK) && t0 != 0 && t0 != p->next_t0)
        return fail(GATEAU_EORDER, "t0=%lld does not continue the previous chunk (next t0 is %lld, or 0 to restart)", t0,
                    p->next_t0);
    if ((p->desc.noise_flags & GATEAU_NOISE_PINK) && p->tk_n > 0 && t0 + nt > p->tk_n)
        return fail(GATEAU_EINVAL, "the exact pink-noise realisation covers %lld samples, run needs %lld", p->tk_n,
                    t0 + nt);
    if (p->scan_kind == GATEAU_SCAN_CUSTOM && t0 + nt > p->n_custom)
        return fail(GATEAU_EINVAL, "custom scan has %lld samples, run needs %lld", p->n_custom, t0 + nt);
    return GATEAU_OK;
}

cudaError_t take_event(gateau_plan* p, cudaEvent_t* e) {
    if (!p->ev_pool.empty()) {
        *e = p->ev_pool.back();
        p->ev_pool.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(e);
}

// Records the start/end events of one phase of the current timed run.
struct PhaseTimer {
    gateau_plan* p;
    cudaStream_t s;
    cudaError_t begin(int ph) {
        if (!p->timing) return cudaSuccess;
        gateau_plan::TimedRun& t = p->timed.back();
        cudaError_t e = take_event(p, &t.ev[ph][0]);
        if (e == cudaSuccess) e = take_event(p, &t.ev[ph][1]);
        if (e != cudaSuccess) return e;
        t.used[ph] = true;
        return cudaEventRecord(t.ev[ph][0], s);
    }
    cudaError_t end(int ph) {
        if (!p->timing) return cudaSuccess;
        return cudaEventRecord(p->timed.back().ev[ph][1], s);
    }
};

// A validated run in three phases, so that a batch can put several plans' contractions into
// shared launches.  Phase 1: derived tables, chunk bookkeeping and the row setup.
gateau_status run_rows(gateau_plan* p, long long t0, long long nt, cudaStream_t stream, bool reset_state = true) {
    gateau_status st = finalize(p);
    if (st != GATEAU_OK) return st;
    const gateau_plan_desc& d = p->desc;
    const long long rows = nt * d.n_pix;
    GATEAU_CUDA(grow(p, p->d_rows, static_cast<size_t>(rows) * sizeof(RowParams)));
    const DevTables T = make_tables(p);
    RowParams* R = p->d_rows.as<RowParams>();
    if (p->timing) {
        gateau_plan::TimedRun t{};
        p->timed.push_back(t);
    }
    PhaseTimer tm{p, stream};
    if (t0 == 0 && reset_state) {
        GATEAU_CUDA(cudaMemsetAsync(p->d_state.p, 0, static_cast<size_t>(d.n_pix) * p->n_ch * p->n_pole * sizeof(float),
                                    stream));
    }
    if (p->cube_scale_dirty) {
        GATEAU_CUDA(launch_scale_cube(p->d_cube_raw.as<float>(), T.c2, static_cast<long long>(p->n_az) * p->n_el,
                                      p->Kp, p->d_cube.as<float>(), stream));
        p->launches += 1;
        p->cube_scale_dirty = false;
    }
    TileInfo* tiles = nullptr;
    if (d.precision == GATEAU_PREC_BF16X3) {
        const long long n_tiles = (nt + kTileRows - 1) / kTileRows * d.n_pix;
        GATEAU_CUDA(grow(p, p->d_tiles, static_cast<size_t>(n_tiles) * sizeof(TileInfo)));
        tiles = p->d_tiles.as<TileInfo>();
        if (p->maps_dirty) {
            std::string err;
            p->fused.tma_inputs = fused_encode_input_maps(p->d_tau.as<float>(), p->n_pwv, p->d_cube.as<float>(),
                                                          p->n_az, p->n_el, p->Kp, &p->tm_tau, &p->tm_tau_s, &p->tm_cube,
                                                          &p->tm_cube_s, err)
                                      ? 1
                                      : 0;
            p->maps_dirty = false;
        }
    }
    GATEAU_CUDA(tm.begin(GATEAU_PHASE_ROWS));
    GATEAU_CUDA(launch_row_setup(T, t0, nt, R, tiles, stream));
    GATEAU_CUDA(tm.end(GATEAU_PHASE_ROWS));
    p->launches += 1;
    return GATEAU_OK;
}

// The split-BF16 contraction of a run, as one job of a fused launch.
FusedRunDesc fused_run(const gateau_plan* p, long long t0, long long nt, float* out) {
    FusedRunDesc r;
    r.T = make_tables(p);
    r.F = p->fused;
    r.tm_tau = p->tm_tau;
    r.tm_tau_s = p->tm_tau_s;
    r.tm_cube = p->tm_cube;
    r.tm_cube_s = p->tm_cube_s;
    r.rows = p->d_rows.as<RowParams>();
    r.tiles = p->d_tiles.as<TileInfo>();
    r.t0 = t0;
    r.nt = nt;
    r.out = out;
    return r;
}

// Phase 2 for one plan alone: the contraction (FP32 baseline, or one fused launch).
gateau_status run_contract(gateau_plan* p, long long t0, long long nt, float* out, cudaStream_t stream) {
    const gateau_plan_desc& d = p->desc;
    PhaseTimer tm{p, stream};
    if (d.precision == GATEAU_PREC_FP32) {
        // Unfused baseline: spectra in HBM chunk by chunk, then the SIMT contraction.
        const DevTables T = make_tables(p);
        const RowParams* R = p->d_rows.as<RowParams>();
        const long long rows = nt * d.n_pix;
        const long long chunk = std::min<long long>(rows, 131072);
        GATEAU_CUDA(grow(p, p->d_X, static_cast<size_t>(chunk) * p->Kp * sizeof(float)));
        // Timing covers the whole chunk loop: SPECTRUM and CONTRACT alternate, so the
        // loop is reported under CONTRACT and SPECTRUM stays zero for this path.
        GATEAU_CUDA(tm.begin(GATEAU_PHASE_CONTRACT));
        for (long long r0 = 0; r0 < rows; r0 += chunk) {
            const long long nr = std::min(chunk, rows - r0);
            GATEAU_CUDA(launch_psd_fp32(T, R, r0, nr, p->d_X.as<float>(), stream));
            GATEAU_CUDA(launch_contract_fp32(T, p->d_X.as<float>(), r0, nr, t0, nt, out, stream));
            p->launches += 2;
        }
        GATEAU_CUDA(tm.end(GATEAU_PHASE_CONTRACT));
    } else {
        const FusedRunDesc r = fused_run(p, t0, nt, out);
        GATEAU_CUDA(tm.begin(GATEAU_PHASE_CONTRACT));
        GATEAU_CUDA(launch_fused_runs(&r, 1, p->n_sm, stream));
        GATEAU_CUDA(tm.end(GATEAU_PHASE_CONTRACT));
        p->launches += 1;
    }
    return GATEAU_OK;
}

// Phase 3: pink noise (Sect. 2.6) and the chunk bookkeeping.
gateau_status run_noise(gateau_plan* p, long long t0, long long nt, float* out, cudaStream_t stream) {
    const gateau_plan_desc& d = p->desc;
    PhaseTimer tm{p, stream};
    if ((d.noise_flags & GATEAU_NOISE_PINK) && p->tk_n > 0) {
        // exact pink noise: the plan's realisation of samples [t0, t0 + nt), added elementwise
        const long long S = static_cast<long long>(d.n_pix) * p->n_ch;
        GATEAU_CUDA(tm.begin(GATEAU_PHASE_PINK));
        GATEAU_CUDA(launch_tk_add(out, p->d_tk.as<float>() + t0 * S, nt * S, stream));
        GATEAU_CUDA(tm.end(GATEAU_PHASE_PINK));
        p->launches += 1;
    } else if (d.noise_flags & GATEAU_NOISE_PINK) {
        const DevTables T = make_tables(p);
        PinkWork W;
        pink_choose_chunks(nt, static_cast<long long>(d.n_pix) * p->n_ch, W.C, W.L);
        GATEAU_CUDA(grow(p, p->d_agg, static_cast<size_t>(W.C) * d.n_pix * p->n_ch * p->n_pole * sizeof(float)));
        W.agg = p->d_agg.as<float>();
        GATEAU_CUDA(tm.begin(GATEAU_PHASE_PINK));
        GATEAU_CUDA(launch_pink(T, p->d_state.as<float>(), W, t0, nt, out, stream));
        GATEAU_CUDA(tm.end(GATEAU_PHASE_PINK));
        p->launches += 3;
    }
    p->runs += 1;
    p->next_t0 = t0 + nt;
    p->last_stream = stream;
    p->ran = true;
    return GATEAU_OK;
}

// Enqueue one validated run.
gateau_status enqueue_run(gateau_plan* p, long long t0, long long nt, float* out, cudaStream_t stream) {
    gateau_status st = run_rows(p, t0, nt, stream);
    if (st == GATEAU_OK) st = run_contract(p, t0, nt, out, stream);
    if (st == GATEAU_OK) st = run_noise(p, t0, nt, out, stream);
    return st;
}

}  // namespace

extern "C" {

const char* gateau_version(void) { return "gateau-b300 1.0 (sm_103a; fp32 SIMT + split-bf16 tcgen05)"; }

const char* gateau_last_error(void) { return g_last_error.c_str(); }

int gateau_device_count(void) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

gateau_status gateau_plan_create(const gateau_plan_desc* desc, gateau_plan** out) {
    if (!out) return fail(GATEAU_EINVAL, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(GATEAU_EINVAL, "desc is NULL");
    const gateau_plan_desc& d = *desc;
    if (d.n_freq < 2 || d.n_freq > (1 << 20)) return fail(GATEAU_EINVAL, "n_freq must be in [2, 2^20]");
    if (!(d.f_lo_hz > 0.0) || !(d.f_hi_hz > d.f_lo_hz)) return fail(GATEAU_EINVAL, "need 0 < f_lo < f_hi");
    if (!(d.f_sample_hz > 0.0)) return fail(GATEAU_EINVAL, "f_sample must be > 0");
    if (d.n_pix < 1 || d.n_pix > (1 << 20) || !d.pix_offsets_rad) return fail(GATEAU_EINVAL, "need n_pix >= 1 and pix_offsets");
    if (!(d.T_atm_K >= 0.0) || !(d.T_cmb_K >= 0.0)) return fail(GATEAU_EINVAL, "temperatures must be >= 0");
    if (!(d.h_column_m > 0.0)) return fail(GATEAU_EINVAL, "h_column must be > 0");
    if (!(d.eta_pb > 0.0) || !(d.delta_al_J >= 0.0)) return fail(GATEAU_EINVAL, "need eta_pb > 0, delta_al >= 0");
    if (d.precision != GATEAU_PREC_FP32 && d.precision != GATEAU_PREC_BF16X3) return fail(GATEAU_EINVAL, "unknown precision");
    if (!(d.pink_f_min_hz > 0.0) || !(d.pink_f_min_hz < 0.5 * d.f_sample_hz))
        return fail(GATEAU_EINVAL, "need 0 < pink_f_min < f_sample/2");
    if (pink_pole_count(d.pink_f_min_hz, d.f_sample_hz) > kMaxPoles)
        return fail(GATEAU_EINVAL, "pink_f_min too low: the filter would need more than %d poles", kMaxPoles);
    std::unique_ptr<gateau_plan> p(new (std::nothrow) gateau_plan());
    if (!p) return fail(GATEAU_ENOMEM, "host allocation failed");
    p->desc = d;
    p->pix_off.assign(d.pix_offsets_rad, d.pix_offsets_rad + 2 * static_cast<size_t>(d.n_pix));
    p->desc.pix_offsets_rad = p->pix_off.data();
    p->nu = make_grid(d.n_freq, d.f_lo_hz, d.f_hi_hz);
    p->w = make_trapezoid(p->nu);
    p->Kp = (d.n_freq + 31) / 32 * 32;
    p->fused.wait_cycles = kDefaultWaitCycles;
    p->fused.ring_b = kDefaultRingB;
    *out = p.release();
    return GATEAU_OK;
}

void gateau_plan_destroy(gateau_plan* plan) { delete plan; }

// Device-side plan buffers that every run needs (pixel offsets, status word).
static gateau_status ensure_base(gateau_plan* p) {
    if (!p->d_pix.p) {
        // offsets [n_pix][2], then [n_pix][4]: tan dphi, tan dth, sin dth, cos dth (the row
        // setup combines them with the scan pointing through the angle-addition identities)
        const int n = p->desc.n_pix;
        std::vector<double> tab(6 * static_cast<size_t>(n));
        for (int i = 0; i < n; ++i) {
            const double dphi = p->pix_off[2 * i], dth = p->pix_off[2 * i + 1];
            tab[2 * i] = dphi;
            tab[2 * i + 1] = dth;
            double* tr = &tab[2 * static_cast<size_t>(n) + 4 * static_cast<size_t>(i)];
            tr[0] = std::tan(dphi);
            tr[1] = std::tan(dth);
            tr[2] = std::sin(dth);
            tr[3] = std::cos(dth);
        }
        // and the same [n_pix][4] trigonometry in float (the row setup's FP32 angle additions)
        std::vector<float> tab_f(4 * static_cast<size_t>(n));
        for (size_t q = 0; q < tab_f.size(); ++q) tab_f[q] = static_cast<float>(tab[2 * static_cast<size_t>(n) + q]);
        GATEAU_CUDA(grow(p, p->d_pix, tab.size() * sizeof(double) + tab_f.size() * sizeof(float)));
        GATEAU_CUDA(cudaMemcpy(p->d_pix.p, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice));
        GATEAU_CUDA(cudaMemcpy(static_cast<char*>(p->d_pix.p) + tab.size() * sizeof(double), tab_f.data(),
                               tab_f.size() * sizeof(float), cudaMemcpyHostToDevice));
        GATEAU_CUDA(grow(p, p->d_status, sizeof(unsigned int)));
        GATEAU_CUDA(cudaMemset(p->d_status.p, 0, sizeof(unsigned int)));
        int dev = 0;
        GATEAU_CUDA(cudaGetDevice(&dev));
        GATEAU_CUDA(cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, dev));
    }
    return GATEAU_OK;
}

gateau_status gateau_set_source_cube(gateau_plan* p, const float* cube, int n_az, int n_el, double az0_rad,
                                     double daz_rad, double el0_rad, double del_rad, int mem) {
    if (!p || !cube) return fail(GATEAU_EINVAL, "plan and cube must be non-NULL");
    if (check_mem(mem) != GATEAU_OK) return GATEAU_EINVAL;
    if (n_az < 2 || n_el < 2 || n_az > 65535 || n_el > 65535) return fail(GATEAU_EINVAL, "cube needs 2 <= n_az, n_el <= 65535");
    if (!(daz_rad > 0.0) || !(del_rad > 0.0)) return fail(GATEAU_EINVAL, "cube grid steps must be > 0");
    if (static_cast<long long>(n_az) * n_el * p->Kp >= (1LL << 31)) return fail(GATEAU_EINVAL, "cube too large (n_az*n_el*n_freq >= 2^31)");
    gateau_status st = ensure_base(p);
    if (st != GATEAU_OK) return st;
    const size_t nf = p->desc.n_freq, Kp = p->Kp;
    const size_t cube_bytes = static_cast<size_t>(n_az) * n_el * Kp * sizeof(float);
    if (p->d_cube.bytes < cube_bytes || p->n_az != n_az || p->n_el != n_el) p->maps_dirty = true;
    GATEAU_CUDA(grow(p, p->d_cube, cube_bytes));
    GATEAU_CUDA(grow(p, p->d_cube_raw, cube_bytes));
    if (Kp != nf) GATEAU_CUDA(cudaMemset(p->d_cube_raw.p, 0, cube_bytes));
    GATEAU_CUDA(cudaMemcpy2D(p->d_cube_raw.p, Kp * sizeof(float), cube, nf * sizeof(float), nf * sizeof(float),
                             static_cast<size_t>(n_az) * n_el, kind_of(mem)));
    p->n_az = n_az;
    p->n_el = n_el;
    p->az0 = az0_rad;
    p->daz = daz_rad;
    p->el0 = el0_rad;
    p->del = del_rad;
    p->has_cube = true;
    p->cube_scale_dirty = true;
    return GATEAU_OK;
}

gateau_status gateau_set_atmosphere_screen(gateau_plan* p, const float* screen, int nx, int ny, double pitch_m,
                                           int is_epl, double pwv0_mm, int mem) {
    if (!p || !screen) return fail(GATEAU_EINVAL, "plan and screen must be non-NULL");
    if (check_mem(mem) != GATEAU_OK) return GATEAU_EINVAL;
    if (nx < 2 || ny < 2 || !(pitch_m > 0.0)) return fail(GATEAU_EINVAL, "screen needs nx, ny >= 2 and pitch > 0");
    gateau_status st = ensure_base(p);
    if (st != GATEAU_OK) return st;
    const size_t n = static_cast<size_t>(nx) * ny;
    GATEAU_CUDA(grow(p, p->d_screen, n * sizeof(float)));
    // PWV values on the host: a PWV screen in host memory is read (and uploaded) in place; an EPL
    // screen is converted first (Eq. 4), a device screen fetched
    std::vector<float> h;
    const float* hv = screen;
    if (is_epl || mem == GATEAU_MEM_DEVICE) {
        st = fetch_floats(screen, n, mem, h);
        if (st != GATEAU_OK) return st;
        if (is_epl)
            for (float& v : h) v = static_cast<float>(static_cast<double>(v) / 6.587 + pwv0_mm);   // Eq. 4
        hv = h.data();
    }
    if (!is_epl && mem == GATEAU_MEM_DEVICE)
        GATEAU_CUDA(cudaMemcpy(p->d_screen.p, screen, n * sizeof(float), cudaMemcpyDeviceToDevice));
    else
        GATEAU_CUDA(cudaMemcpy(p->d_screen.p, hv, n * sizeof(float), cudaMemcpyHostToDevice));
    double sum = 0.0;                  // the reference spectrum's PWV
    for (size_t i = 0; i < n; ++i) sum += hv[i];
    const double mean = sum / static_cast<double>(n);
    if (!p->has_screen || mean != p->screen_mean) {
        p->ref_dirty = true;
        if (p->pink_auto) p->dirty = true;   // the automatic pink level follows the reference sky
    }
    p->screen_mean = mean;
    p->nx = nx;
    p->ny = ny;
    p->pitch = pitch_m;
    p->has_screen = true;
    return GATEAU_OK;
}

gateau_status gateau_set_atmosphere_table(gateau_plan* p, const float* table, int n_pwv, double pwv_min_mm,
                                          double dpwv_mm, int is_opacity, int mem) {
    if (!p || !table) return fail(GATEAU_EINVAL, "plan and table must be non-NULL");
    if (check_mem(mem) != GATEAU_OK) return GATEAU_EINVAL;
    if (n_pwv < 2 || !(dpwv_mm > 0.0)) return fail(GATEAU_EINVAL, "table needs n_pwv >= 2 and dpwv > 0");
    gateau_status st = ensure_base(p);
    if (st != GATEAU_OK) return st;
    const size_t nf = p->desc.n_freq, Kp = p->Kp, n = static_cast<size_t>(n_pwv) * nf;
    std::vector<float> h;
    const float* hv = table;                // the values on the host: in place, or fetched from the device
    if (mem == GATEAU_MEM_DEVICE) {
        st = fetch_floats(table, n, mem, h);
        if (st != GATEAU_OK) return st;
        hv = h.data();
    }
    // The table is checked and kept (the reference spectrum converts the two rows it reads to FP64)
    // only when its values change; the device rows are uploaded on every call.
    const bool same = p->has_table && p->n_pwv == n_pwv && p->table_is_opacity == (is_opacity != 0) &&
                      p->table_raw.size() == n && memcmp(p->table_raw.data(), hv, n * sizeof(float)) == 0;
    std::vector<float> tf;                  // a transmission table's opacities rounded to float
    if (!same) {
        if (is_opacity) {
            bool ok = true;                 // NaN fails v >= 0, +inf fails v <= FLT_MAX
            for (size_t i = 0; i < n; ++i) ok &= (hv[i] >= 0.f) & (hv[i] <= FLT_MAX);
            if (!ok)
                for (size_t i = 0; i < n; ++i)
                    if (!(hv[i] >= 0.f && hv[i] <= FLT_MAX))
                        return fail(GATEAU_EINVAL, "opacity must be finite and >= 0 (row %zu, point %zu)", i / nf, i % nf);
        } else {
            tf.resize(n);
            for (size_t i = 0; i < n; ++i) {
                const double v = -log(std::max(static_cast<double>(hv[i]), 1e-30));
                if (!(v >= 0.0) || !std::isfinite(v))
                    return fail(GATEAU_EINVAL, "opacity must be finite and >= 0 (row %zu, point %zu)", i / nf, i % nf);
                tf[i] = static_cast<float>(v);
            }
        }
        p->ref_dirty = true;
        if (p->pink_auto) p->dirty = true;
        p->table_raw.assign(hv, hv + n);
        p->table_is_opacity = is_opacity != 0;
    }
    if (pwv_min_mm != p->pwv_min || dpwv_mm != p->dpwv) {
        p->ref_dirty = true;                 // the reference PWV's row moves
        if (p->pink_auto) p->dirty = true;
    }
    // Device: the rows tau_j as float (an opacity table is that already), then interleaved
    // [n_pwv][2][Kp] -- row 2j tau_j, row 2j+1 tau_{j+1} - tau_j (0 for the last j) -- by a kernel.
    GATEAU_CUDA(grow(p, p->d_tau_rows, n * sizeof(float)));
    GATEAU_CUDA(grow(p, p->d_tau, static_cast<size_t>(2 * n_pwv) * Kp * sizeof(float)));
    if (is_opacity) {
        GATEAU_CUDA(cudaMemcpy(p->d_tau_rows.p, table, n * sizeof(float), kind_of(mem)));
    } else {
        if (same) {                         // unchanged transmissions: round the kept table again
            tf.resize(n);
            for (size_t i = 0; i < n; ++i) tf[i] = static_cast<float>(table_opacity(p, i));
        }
        GATEAU_CUDA(cudaMemcpy(p->d_tau_rows.p, tf.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    }
    GATEAU_CUDA(launch_tau_interleave(p->d_tau_rows.as<float>(), n_pwv, static_cast<int>(nf), static_cast<int>(Kp),
                                      p->d_tau.as<float>(), nullptr));
    GATEAU_CUDA(cudaStreamSynchronize(nullptr));
    p->n_pwv = n_pwv;
    p->pwv_min = pwv_min_mm;
    p->dpwv = dpwv_mm;
    p->has_table = true;
    p->maps_dirty = true;
    if (p->kelvin) p->dirty = true;    // the skydip reads the table
    return GATEAU_OK;
}

gateau_status gateau_set_cascade(gateau_plan* p, int n_stage, const gateau_stage* stages) {
    if (!p) return fail(GATEAU_EINVAL, "plan is NULL");
    if (n_stage < 0 || n_stage > 64 || (n_stage > 0 && !stages)) return fail(GATEAU_EINVAL, "need 0 <= n_stage <= 64 and stages");
    std::vector<StageSpec> v;
    for (int s = 0; s < n_stage; ++s) {
        const gateau_stage& g = stages[s];
        StageSpec st{};
        st.kind = g.kind;
        st.T_K = g.T_K;
        st.eta = g.eta;
        if (g.kind == GATEAU_STAGE_REFLECTIVE && g.eta_nu) st.eta_nu.assign(g.eta_nu, g.eta_nu + p->desc.n_freq);
        st.eps_ref = g.eps_ref;
        st.nu_ref_hz = g.nu_ref_hz;
        st.d_m = g.d_m;
        st.n_index = g.n_index;
        st.tan_delta = g.tan_delta;
        st.T_refl_K = g.T_refl_K;
        st.ar_coated = g.ar_coated;
        v.push_back(std::move(st));
    }
    std::vector<PrimStage> prim;
    std::string err;
    if (!expand_stages(v, p->nu, prim, err)) return fail(GATEAU_EINVAL, "%s", err.c_str());
    p->stages = std::move(v);
    p->has_cascade = true;
    p->dirty = true;
    return GATEAU_OK;
}

gateau_status gateau_set_dispersive_element(gateau_plan* p, int kind, int n_ch, const double* f_c_hz, const double* R,
                                            const double* eta_peak, const double* custom_eta) {
    if (!p) return fail(GATEAU_EINVAL, "plan is NULL");
    if (n_ch < 1 || n_ch > 4096) return fail(GATEAU_EINVAL, "need 1 <= n_ch <= 4096");
    std::vector<double> eta;
    std::string err;
    if (!build_filters(kind, n_ch, f_c_hz, R, eta_peak, custom_eta, p->nu, p->desc.delta_al_J, eta, err))
        return fail(GATEAU_EINVAL, "%s", err.c_str());
    if (p->has_disp && n_ch != p->n_ch) {
        p->has_pink = false;
        p->track_streams();
        p->d_state.release(p->mo);
    }
    p->eta_filt = std::move(eta);
    p->disp_kind = kind;
    p->n_ch = n_ch;
    p->has_disp = true;
    p->dirty = true;
    return GATEAU_OK;
}

gateau_status gateau_set_pink_noise(gateau_plan* p, const double* A, const double* alpha) {
    if (!p || !alpha) return fail(GATEAU_EINVAL, "plan and alpha must be non-NULL");
    if (!p->has_disp) return fail(GATEAU_ESTATE, "set the dispersive element before the pink noise");
    for (int c = 0; c < p->n_ch; ++c)
        if ((A && !(A[c] >= 0.0)) || !(alpha[c] >= 0.0 && alpha[c] <= 3.0))
            return fail(GATEAU_EINVAL, "channel %d: need A >= 0 and 0 <= alpha <= 3", c);
    p->pink_auto = A == nullptr;
    if (A) p->pink_A.assign(A, A + p->n_ch);
    else p->pink_A.assign(p->n_ch, 0.0);          // set from the reference spectrum when prepared
    p->pink_alpha.assign(alpha, alpha + p->n_ch);
    p->has_pink = true;
    p->dirty = true;
    return GATEAU_OK;
}

gateau_status gateau_set_scan(gateau_plan* p, int kind, const double* params, int n_params, double phi0_rad,
                              double theta0_rad, const double* custom, long long n_custom, int mem) {
    if (!p) return fail(GATEAU_EINVAL, "plan is NULL");
    static const int need[] = {0, 3, 4, 0};
    if (kind < GATEAU_SCAN_STARE || kind > GATEAU_SCAN_CUSTOM) return fail(GATEAU_EINVAL, "unknown scan kind");
    if (n_params < need[kind] || n_params > kMaxScanParams || (n_params > 0 && !params))
        return fail(GATEAU_EINVAL, "scan kind %d needs %d parameters", kind, need[kind]);
    if (kind == GATEAU_SCAN_RASTER && (!(params[0] > 0.0) || !(params[1] > 0.0) || params[3] < 1.0))
        return fail(GATEAU_EINVAL, "raster needs half_width > 0, speed > 0, n_rows >= 1");
    if (kind == GATEAU_SCAN_CUSTOM) {
        if (!custom || n_custom < 1) return fail(GATEAU_EINVAL, "custom scan needs a pointing table");
        if (check_mem(mem) != GATEAU_OK) return GATEAU_EINVAL;
        gateau_status st = ensure_base(p);
        if (st != GATEAU_OK) return st;
        GATEAU_CUDA(grow(p, p->d_custom, static_cast<size_t>(n_custom) * 2 * sizeof(double)));
        GATEAU_CUDA(cudaMemcpy(p->d_custom.p, custom, static_cast<size_t>(n_custom) * 2 * sizeof(double), kind_of(mem)));
    }
    p->scan_kind = kind;
    for (int i = 0; i < kMaxScanParams; ++i) p->sp[i] = i < n_params ? params[i] : 0.0;
    p->phi0 = phi0_rad;
    if (!p->has_scan || theta0_rad != p->theta0) {   // the reference spectrum's elevation
        p->ref_dirty = true;
        if (p->pink_auto) p->dirty = true;
    }
    p->theta0 = theta0_rad;
    p->n_custom = kind == GATEAU_SCAN_CUSTOM ? n_custom : 0;
    if (p->kelvin) p->dirty = true;    // the skydip runs at the base elevation theta0
    p->has_scan = true;
    return GATEAU_OK;
}

gateau_status gateau_set_output_kelvin(gateau_plan* p, int enable, double pwv_lo_mm, double pwv_hi_mm, int n_pwv) {
    if (!p) return fail(GATEAU_EINVAL, "plan must be non-NULL");
    if (enable) {
        if (n_pwv < 2 || n_pwv > kMaxSkydip) return fail(GATEAU_EINVAL, "skydip needs 2 <= n_pwv <= %d", kMaxSkydip);
        if (!std::isfinite(pwv_lo_mm) || !std::isfinite(pwv_hi_mm) || !(pwv_lo_mm < pwv_hi_mm) || pwv_lo_mm < 0.0)
            return fail(GATEAU_EINVAL, "skydip needs 0 <= pwv_lo < pwv_hi (finite)");
    }
    p->kelvin = enable != 0;
    p->dip_lo = pwv_lo_mm;
    p->dip_hi = pwv_hi_mm;
    p->dip_n = n_pwv;
    p->dirty = true;
    return GATEAU_OK;
}

gateau_status gateau_set_pink_timmer_koenig(gateau_plan* p, long long n_total) {
    if (!p) return fail(GATEAU_EINVAL, "plan must be non-NULL");
    if (n_total < 0 || n_total > (1LL << 30)) return fail(GATEAU_EINVAL, "need 0 <= n_total <= 2^30 (got %lld)", n_total);
    p->tk_n = n_total;
    p->dirty = true;
    return GATEAU_OK;
}

gateau_status gateau_mean_zenith_pwv(gateau_plan* p, long long n_total, double* pwv_mean_mm) {
    if (!p || !pwv_mean_mm) return fail(GATEAU_EINVAL, "plan and pwv_mean_mm must be non-NULL");
    gateau_status st = check_complete(p);
    if (st != GATEAU_OK) return st;
    if (n_total <= 0) return fail(GATEAU_EINVAL, "need n_total > 0");
    if (p->scan_kind == GATEAU_SCAN_CUSTOM && n_total > p->n_custom)
        return fail(GATEAU_EINVAL, "custom scan has %lld samples, the mean needs %lld", p->n_custom, n_total);
    st = finalize(p);
    if (st != GATEAU_OK) return st;
    const int n_pix = p->desc.n_pix;
    const long long chunk = std::max<long long>(1, (1LL << 22) / n_pix);
    GATEAU_CUDA(grow(p, p->d_rows, static_cast<size_t>(std::min(chunk, n_total)) * n_pix * sizeof(RowParams)));
    GATEAU_CUDA(grow(p, p->d_cm, 64));
    double* sum = p->d_cm.as<double>();
    GATEAU_CUDA(cudaMemset(sum, 0, sizeof(double)));
    const DevTables T = make_tables(p);
    for (long long t0 = 0; t0 < n_total; t0 += chunk) {
        const long long nt = std::min(chunk, n_total - t0);
        GATEAU_CUDA(launch_row_setup(T, t0, nt, p->d_rows.as<RowParams>(), nullptr, nullptr));
        GATEAU_CUDA(launch_sum_pwv(p->d_rows.as<RowParams>(), nt * n_pix, sum, nullptr));
        p->launches += 2;
    }
    double h = 0.0;
    GATEAU_CUDA(cudaMemcpy(&h, sum, sizeof(double), cudaMemcpyDeviceToHost));
    *pwv_mean_mm = h / (static_cast<double>(n_total) * n_pix);
    return GATEAU_OK;
}

gateau_status gateau_common_mode(gateau_plan* p, long long t0, long long nt, const float* tb, float* out,
                                 double pwv_mean_mm, double r_out_rad, void* stream) {
    if (!p || !tb || !out) return fail(GATEAU_EINVAL, "plan, tb and out must be non-NULL");
    gateau_status st = check_complete(p);
    if (st != GATEAU_OK) return st;
    if (t0 < 0 || nt <= 0) return fail(GATEAU_EINVAL, "need t0 >= 0 and nt > 0");
    if (nt > (1LL << 31) / p->desc.n_pix) return fail(GATEAU_EINVAL, "nt * n_pix must stay below 2^31");
    if (t0 > (1LL << 62)) return fail(GATEAU_EINVAL, "t0 must stay below 2^62");
    if (!std::isfinite(pwv_mean_mm) || !std::isfinite(r_out_rad)) return fail(GATEAU_EINVAL, "non-finite argument");
    if (p->scan_kind == GATEAU_SCAN_CUSTOM && t0 + nt > p->n_custom)
        return fail(GATEAU_EINVAL, "custom scan has %lld samples, the reduction needs %lld", p->n_custom, t0 + nt);
    const int n_pix = p->desc.n_pix, n_ch = p->n_ch, nf = p->desc.n_freq;
    // S_j (Eq. 26): spaxels farther than r_out from the IFU centre
    std::vector<unsigned char> off(n_pix, 0);
    int n_out = 0;
    for (int j = 0; j < n_pix; ++j)
        if (std::hypot(p->pix_off[2 * j], p->pix_off[2 * j + 1]) > r_out_rad) {
            off[j] = 1;
            ++n_out;
        }
    if (n_out == 0) return fail(GATEAU_EINVAL, "no spaxel lies farther than r_out = %g rad from the centre", r_out_rad);
    st = finalize(p);
    if (st != GATEAU_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t hw_n = static_cast<size_t>(n_ch) * nf;
    if (p->d_hw.bytes < hw_n * sizeof(double)) {
        std::vector<double> hw(hw_n);
        for (int c = 0; c < n_ch; ++c)
            for (int k = 0; k < nf; ++k) hw[static_cast<size_t>(c) * nf + k] = p->eta_filt[static_cast<size_t>(c) * nf + k] * p->w[k];
        GATEAU_CUDA(grow(p, p->d_hw, hw_n * sizeof(double)));
        GATEAU_CUDA(cudaMemcpy(p->d_hw.p, hw.data(), hw_n * sizeof(double), cudaMemcpyHostToDevice));
    }
    GATEAU_CUDA(grow(p, p->d_cm, 64 + static_cast<size_t>(n_ch) * sizeof(float) + n_pix));
    float* log_eta = reinterpret_cast<float*>(p->d_cm.as<uint8_t>() + 64);
    unsigned char* d_off = reinterpret_cast<unsigned char*>(log_eta + n_ch);
    GATEAU_CUDA(cudaMemcpyAsync(d_off, off.data(), n_pix, cudaMemcpyHostToDevice, s));
    GATEAU_CUDA(grow(p, p->d_rows, static_cast<size_t>(nt) * n_pix * sizeof(RowParams)));
    const DevTables T = make_tables(p);
    GATEAU_CUDA(launch_band_transmission(p->d_hw.as<double>(), p->d_tau.as<float>(), nf, p->Kp, p->n_pwv, p->pwv_min,
                                         p->dpwv, pwv_mean_mm, n_ch, log_eta, s));
    GATEAU_CUDA(launch_row_setup(T, t0, nt, p->d_rows.as<RowParams>(), nullptr, s));
    GATEAU_CUDA(launch_common_mode(tb, out, p->d_rows.as<RowParams>(), nt, n_pix, n_ch, log_eta, d_off, n_out, s));
    p->launches += 3;
    p->last_stream = s;
    p->ran = true;
    return GATEAU_OK;
}

// ---- preprocessing utilities (Sect. 2.2, Eqs. 1-3): scratch in the stream-ordered pool of `stream` ----
static bool pow2(int n) { return n >= 2 && (n & (n - 1)) == 0; }

static gateau_status check_beam(double d_az, double d_el, double R, double t_edge) {
    if (!(d_az > 0.0) || !(d_el > 0.0) || !(R > 0.0) || !std::isfinite(d_az) || !std::isfinite(d_el) ||
        !std::isfinite(R) || !std::isfinite(t_edge))
        return fail(GATEAU_EINVAL, "need pitches > 0, R_tel > 0 and a finite edge taper");
    return GATEAU_OK;
}

gateau_status gateau_beam_far_field(const double* nu_hz, int n_freq, int n_a, int n_e, double d_az_rad, double d_el_rad,
                                    double R_tel_m, double t_edge_db, float* dev_F, void* stream) {
    if (!nu_hz || !dev_F) return fail(GATEAU_EINVAL, "nu_hz and dev_F must be non-NULL");
    if (n_freq < 1 || !pow2(n_a) || !pow2(n_e)) return fail(GATEAU_EINVAL, "need n_freq >= 1 and n_a, n_e powers of two >= 2");
    if (check_beam(d_az_rad, d_el_rad, R_tel_m, t_edge_db) != GATEAU_OK) return GATEAU_EINVAL;
    for (int k = 0; k < n_freq; ++k)
        if (!(nu_hz[k] > 0.0) || !std::isfinite(nu_hz[k])) return fail(GATEAU_EINVAL, "frequencies must be > 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long plane = static_cast<long long>(n_a) * n_e;
    // frequencies per batch (also the transposes' grid z extent, <= 65535)
    const int B = static_cast<int>(std::max<long long>(1, std::min<long long>({n_freq, (1LL << 24) / plane, 4096LL})));
    void *dnu = nullptr, *buf = nullptr;
    GATEAU_CUDA(cudaMallocAsync(&dnu, n_freq * sizeof(double), s));
    if (cudaError_t ea = cudaMallocAsync(&buf, 2 * static_cast<size_t>(B) * plane * sizeof(float2) + B * sizeof(float), s);
        ea != cudaSuccess) {
        cudaFreeAsync(dnu, s);
        GATEAU_CUDA(ea);
    }
    float2* F = static_cast<float2*>(buf);
    float2* work = F + static_cast<size_t>(B) * plane;
    float* peak = reinterpret_cast<float*>(work + static_cast<size_t>(B) * plane);
    cudaError_t e = cudaMemcpyAsync(dnu, nu_hz, n_freq * sizeof(double), cudaMemcpyHostToDevice, s);
    for (int f0 = 0; f0 < n_freq && e == cudaSuccess; f0 += B) {
        const int b = std::min(B, n_freq - f0);
        e = launch_beam_planes(static_cast<double*>(dnu) + f0, b, n_a, n_e, d_az_rad, d_el_rad, R_tel_m, t_edge_db, F,
                               work, peak, s);
        if (e == cudaSuccess) e = launch_real_part(F, dev_F + static_cast<size_t>(f0) * plane, b * plane, s);
    }
    cudaStreamSynchronize(s);     // nu_hz is the caller's pageable memory
    cudaFreeAsync(buf, s);
    cudaFreeAsync(dnu, s);
    GATEAU_CUDA(e);
    return GATEAU_OK;
}

gateau_status gateau_convolve_source(const float* dev_I, int n_az, int n_el, int n_freq, const double* nu_hz,
                                     double el0_rad, double d_az_rad, double d_el_rad, double R_tel_m, double t_edge_db,
                                     float* dev_P, void* stream) {
    if (!dev_I || !dev_P || !nu_hz) return fail(GATEAU_EINVAL, "dev_I, dev_P and nu_hz must be non-NULL");
    if (dev_I == dev_P) return fail(GATEAU_EINVAL, "dev_P must not alias dev_I");
    if (n_freq < 1 || !pow2(n_az) || !pow2(n_el)) return fail(GATEAU_EINVAL, "need n_freq >= 1 and n_az, n_el powers of two >= 2");
    if (check_beam(d_az_rad, d_el_rad, R_tel_m, t_edge_db) != GATEAU_OK || !std::isfinite(el0_rad)) return GATEAU_EINVAL;
    for (int k = 0; k < n_freq; ++k)
        if (!(nu_hz[k] > 0.0) || !std::isfinite(nu_hz[k])) return fail(GATEAU_EINVAL, "frequencies must be > 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long plane = 4LL * n_az * n_el;
    const int B = static_cast<int>(std::max<long long>(1, std::min<long long>({n_freq, (1LL << 23) / plane, 4096LL})));
    void *dnu = nullptr, *buf = nullptr;
    GATEAU_CUDA(cudaMallocAsync(&dnu, n_freq * sizeof(double), s));
    if (cudaError_t ea = cudaMallocAsync(&buf, 3 * static_cast<size_t>(B) * plane * sizeof(float2) + B * sizeof(float), s);
        ea != cudaSuccess) {
        cudaFreeAsync(dnu, s);
        GATEAU_CUDA(ea);
    }
    float2* K = static_cast<float2*>(buf);
    float2* S = K + static_cast<size_t>(B) * plane;
    float2* work = S + static_cast<size_t>(B) * plane;
    float* peak = reinterpret_cast<float*>(work + static_cast<size_t>(B) * plane);
    cudaError_t e = cudaMemcpyAsync(dnu, nu_hz, n_freq * sizeof(double), cudaMemcpyHostToDevice, s);
    for (int f0 = 0; f0 < n_freq && e == cudaSuccess; f0 += B)
        e = launch_convolve_source_batch(dev_I, dev_P, static_cast<double*>(dnu), std::min(B, n_freq - f0), f0, n_freq,
                                         n_az, n_el, el0_rad, d_az_rad, d_el_rad, R_tel_m, t_edge_db, K, S, work, peak, s);
    cudaStreamSynchronize(s);
    cudaFreeAsync(buf, s);
    cudaFreeAsync(dnu, s);
    GATEAU_CUDA(e);
    return GATEAU_OK;
}

gateau_status gateau_smooth_screen(const float* dev_screen, int nx, int ny, double pitch_m, double R_tel_m,
                                   double t_edge_db, float* dev_out, void* stream) {
    if (!dev_screen || !dev_out) return fail(GATEAU_EINVAL, "dev_screen and dev_out must be non-NULL");
    if (!pow2(nx) || !pow2(ny)) return fail(GATEAU_EINVAL, "need nx, ny powers of two >= 2");
    if (check_beam(pitch_m, pitch_m, R_tel_m, t_edge_db) != GATEAU_OK) return GATEAU_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = static_cast<size_t>(nx) * ny;
    void* buf = nullptr;
    GATEAU_CUDA(cudaMallocAsync(&buf, 3 * n * sizeof(float2) + sizeof(double), s));
    float2* K = static_cast<float2*>(buf);
    cudaError_t e = launch_smooth_screen(dev_screen, dev_out, nx, ny, pitch_m, R_tel_m, t_edge_db, K, K + n, K + 2 * n,
                                         reinterpret_cast<double*>(K + 3 * n), s);
    cudaFreeAsync(buf, s);
    GATEAU_CUDA(e);
    return GATEAU_OK;
}

gateau_status gateau_plan_prepare(gateau_plan* p) {
    if (!p) return fail(GATEAU_EINVAL, "plan is NULL");
    gateau_status st = check_complete(p);
    if (st != GATEAU_OK) return st;
    st = ensure_base(p);
    if (st != GATEAU_OK) return st;
    return finalize(p);
}

gateau_status gateau_run(gateau_plan* p, long long t0, long long nt, float* dev_out, void* stream) {
    if (!p) return fail(GATEAU_EINVAL, "plan is NULL");
    gateau_status st = validate_run(p, t0, nt, dev_out);
    if (st != GATEAU_OK) return st;
    st = ensure_base(p);
    if (st != GATEAU_OK) return st;
    return enqueue_run(p, t0, nt, dev_out, static_cast<cudaStream_t>(stream));
}

gateau_status gateau_run_host(gateau_plan* p, long long t0, long long nt, float* host_out, void* stream) {
    if (!p) return fail(GATEAU_EINVAL, "plan is NULL");
    gateau_status st = validate_run(p, t0, nt, host_out);
    if (st != GATEAU_OK) return st;
    st = ensure_base(p);
    if (st != GATEAU_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!p->copy_stream) {
        GATEAU_CUDA(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
            GATEAU_CUDA(cudaEventCreateWithFlags(&p->ev_done[i], cudaEventDisableTiming));
            GATEAU_CUDA(cudaEventCreateWithFlags(&p->ev_copied[i], cudaEventDisableTiming));
        }
    }
    // Chunks of about 256 MB of output, double-buffered: chunk c runs on `s`
    // while chunk c-1 is copied to the host on the copy stream.  The copies are the
    // slower side, so the first chunk is an eighth as long: the link starts sooner.
    const long long per_sample = static_cast<long long>(p->desc.n_pix) * std::max(p->n_ch, 1);
    const long long chunk = std::max<long long>(128, std::min<long long>(nt, (256LL << 20) / (4 * per_sample)) / 128 * 128);
    const long long first = std::max<long long>(128, chunk / 8 / 128 * 128);
    const size_t chunk_bytes = static_cast<size_t>(std::min(chunk, nt)) * per_sample * sizeof(float);
    for (int i = 0; i < 2; ++i) GATEAU_CUDA(grow(p, p->d_stage[i], chunk_bytes));
    int c = 0;
    for (long long a = 0, len = 0; a < nt; a += len, ++c) {
        const int b = c & 1;
        len = std::min(c == 0 ? first : chunk, nt - a);
        if (c >= 2) GATEAU_CUDA(cudaStreamWaitEvent(s, p->ev_copied[b], 0));
        st = enqueue_run(p, t0 + a, len, p->d_stage[b].as<float>(), s);
        if (st != GATEAU_OK) return st;
        GATEAU_CUDA(cudaEventRecord(p->ev_done[b], s));
        GATEAU_CUDA(cudaStreamWaitEvent(p->copy_stream, p->ev_done[b], 0));
        GATEAU_CUDA(cudaMemcpyAsync(host_out + a * per_sample, p->d_stage[b].p,
                                    static_cast<size_t>(len) * per_sample * sizeof(float), cudaMemcpyDeviceToHost,
                                    p->copy_stream));
        GATEAU_CUDA(cudaEventRecord(p->ev_copied[b], p->copy_stream));
    }
    GATEAU_CUDA(cudaStreamSynchronize(p->copy_stream));
    GATEAU_CUDA(cudaStreamSynchronize(s));
    return GATEAU_OK;
}

gateau_status gateau_run_batch(gateau_plan* const* plans, const long long* t0s, const long long* nts, float* const* outs,
                               int n, void* stream) {
    if (!plans || !t0s || !nts || !outs || n <= 0 || n > 256) return fail(GATEAU_EINVAL, "need 0 < n <= 256 and arrays");
    for (int k = 0; k < n; ++k) {
        if (!plans[k]) return fail(GATEAU_EINVAL, "plans[%d] is NULL", k);
        for (int m = 0; m < k; ++m)
            if (plans[m] == plans[k]) return fail(GATEAU_EINVAL, "plan %d appears twice in the batch", k);
        gateau_status st = validate_run(plans[k], t0s[k], nts[k], outs[k]);
        if (st != GATEAU_OK) return st;
        st = ensure_base(plans[k]);
        if (st != GATEAU_OK) return st;
    }
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    for (int k = 0; k < n; ++k) {
        gateau_status st = run_rows(plans[k], t0s[k], nts[k], cs);
        if (st != GATEAU_OK) return st;
    }
    // The FP32 baseline runs plan by plan; the split-BF16 contractions of the batch share
    // persistent launches, one per launch mode (shared tiles for two channel groups, independent
    // CTAs otherwise) and per fused_max_jobs() plans.
    std::vector<int> mode[2];
    for (int k = 0; k < n; ++k) {
        gateau_plan* p = plans[k];
        if (p->desc.precision == GATEAU_PREC_FP32) {
            gateau_status st = run_contract(p, t0s[k], nts[k], outs[k], cs);
            if (st != GATEAU_OK) return st;
        } else {
            mode[p->fused.n_groups == 2 ? 1 : 0].push_back(k);
        }
    }
    for (const std::vector<int>& ks : mode)
        for (size_t a = 0; a < ks.size(); a += static_cast<size_t>(fused_max_jobs())) {
            const size_t b = std::min(ks.size(), a + static_cast<size_t>(fused_max_jobs()));
            std::vector<FusedRunDesc> runs;
            for (size_t i = a; i < b; ++i) runs.push_back(fused_run(plans[ks[i]], t0s[ks[i]], nts[ks[i]], outs[ks[i]]));
            for (size_t i = a; i < b; ++i) GATEAU_CUDA((PhaseTimer{plans[ks[i]], cs}.begin(GATEAU_PHASE_CONTRACT)));
            GATEAU_CUDA(launch_fused_runs(runs.data(), static_cast<int>(runs.size()), plans[ks[a]]->n_sm, cs));
            for (size_t i = a; i < b; ++i) GATEAU_CUDA((PhaseTimer{plans[ks[i]], cs}.end(GATEAU_PHASE_CONTRACT)));
            plans[ks[a]]->launches += 1;          // one launch for the whole group, counted once
        }
    for (int k = 0; k < n; ++k) {
        gateau_status st = run_noise(plans[k], t0s[k], nts[k], outs[k], cs);
        if (st != GATEAU_OK) return st;
    }
    return GATEAU_OK;
}

gateau_status gateau_plan_estimate_bytes(const gateau_plan_desc* d, int n_ch, int n_az, int n_el, int nx, int ny,
                                         int n_pwv, long long chunk, long long n_custom, size_t* bytes) {
    if (!d || !bytes) return fail(GATEAU_EINVAL, "desc and bytes must be non-NULL");
    *bytes = 0;
    if (d->n_freq < 2 || d->n_pix < 1 || n_ch < 1 || n_az < 2 || n_el < 2 || nx < 1 || ny < 1 || n_pwv < 2 ||
        chunk < 1 || n_custom < 0)
        return fail(GATEAU_EINVAL, "need n_freq >= 2, n_pix, n_ch, nx, ny, chunk >= 1, cube and table >= 2");
    if (!(d->pink_f_min_hz > 0.0) || !(d->f_sample_hz > 2.0 * d->pink_f_min_hz))
        return fail(GATEAU_EINVAL, "need 0 < pink_f_min < f_sample/2");
    const double Kp = static_cast<double>((d->n_freq + 31) / 32 * 32);
    const int np = pink_pole_count(d->pink_f_min_hz, d->f_sample_hz);
    const double n_pix = d->n_pix, nc = n_ch;
    double b = n_pix * (6 * 8 + 4 * 4) + 64;                         // spaxel offsets and trig, status word
    b += 2.0 * n_az * n_el * Kp * 4;                                 // source cube as set + scaled copy
    b += static_cast<double>(nx) * ny * 4;                           // screen
    b += 2.0 * n_pwv * Kp * 4 + static_cast<double>(n_pwv) * d->n_freq * 4;   // interleaved opacity table + its rows as set
    b += 5.0 * Kp * 4;                                               // c0, c1, c2 + per-stage tiling
    if (d->precision == GATEAU_PREC_FP32) {
        b += 3.0 * ((n_ch + 63) / 64 * 64) * Kp * 4;                 // FP32 H, G, Q
        b += std::min(static_cast<double>(chunk) * n_pix, 131072.0) * Kp * 4;   // spectrum chunk
    } else {
        const int n_groups = (n_ch + 175) / 176;   // groups of <= 176 channels: B stages fit the rings
        const int n_half = ((n_ch + n_groups - 1) / n_groups + 15) / 16 * 16;
        b += static_cast<double>(n_groups) * n_half * 4 * Kp * 2;    // BF16 operands
        b += std::ceil(static_cast<double>(chunk) / kTileRows) * n_pix * sizeof(TileInfo);
    }
    b += nc * (2 * np + 1) * 4 + n_pix * nc * np * 4;                // pink tables + state
    b += static_cast<double>(chunk) * n_pix * sizeof(RowParams);     // row parameters
    int C = 1;
    long long L = chunk;
    pink_choose_chunks(chunk, static_cast<long long>(d->n_pix) * n_ch, C, L);
    b += static_cast<double>(C) * n_pix * nc * np * 4;               // pink chunk states
    b += static_cast<double>(n_custom) * 2 * 8;                      // custom pointing
    b += 24 * 4096;                                                  // allocation granularity
    *bytes = static_cast<size_t>(b);
    return GATEAU_OK;
}

gateau_status gateau_plan_status(gateau_plan* p, unsigned int* flags) {
    if (!p || !flags) return fail(GATEAU_EINVAL, "plan and flags must be non-NULL");
    *flags = 0;
    if (!p->d_status.p) return GATEAU_OK;
    GATEAU_CUDA(cudaStreamSynchronize(p->last_stream));
    GATEAU_CUDA(cudaMemcpy(flags, p->d_status.p, sizeof(unsigned int), cudaMemcpyDeviceToHost));
    GATEAU_CUDA(cudaMemset(p->d_status.p, 0, sizeof(unsigned int)));
    if (*flags & GATEAU_STATUS_WAIT_TIMEOUT) return fail(GATEAU_ETIMEOUT, "a fused-kernel pipeline wait timed out");
    if (*flags & ~static_cast<unsigned int>(GATEAU_STATUS_PWV_CLAMPED))
        return fail(GATEAU_EDEVICE, "device status word 0x%x", *flags);
    return GATEAU_OK;
}

gateau_status gateau_plan_get_info(gateau_plan* p, gateau_plan_info* info) {
    if (!p || !info) return fail(GATEAU_EINVAL, "plan and info must be non-NULL");
    info->n_freq = p->desc.n_freq;
    info->n_freq_padded = p->Kp;
    info->n_ch = p->n_ch;
    info->n_pix = p->desc.n_pix;
    info->n_pole = pink_pole_count(p->desc.pink_f_min_hz, p->desc.f_sample_hz);
    info->next_t0 = p->next_t0;
    info->device_bytes = device_bytes(p);
    info->staged_inputs = p->fused.tma_inputs;
    info->tile_groups = info->tile_half = info->ring_a = info->ring_b = 0;
    if (p->desc.precision == GATEAU_PREC_BF16X3 && p->fused.n_half > 0) {
        info->tile_groups = p->fused.n_groups;
        info->tile_half = p->fused.n_half;
        info->ring_b = fused_ring_depths(p->fused.n_half, p->fused.ring_b, &info->ring_a);
    }
    info->tune_ms = p->tune_ms;
    return GATEAU_OK;
}

gateau_status gateau_plan_get_vector(gateau_plan* p, int which, double* out, size_t count) {
    if (!p || !out) return fail(GATEAU_EINVAL, "plan and out must be non-NULL");
    const std::vector<double>* src = nullptr;
    std::vector<double> tmp;
    const bool needs_tables = which >= GATEAU_VEC_C0 && which <= GATEAU_VEC_PINK_D;
    if (which == GATEAU_VEC_ETA_FILT && !p->has_disp) return fail(GATEAU_ESTATE, "dispersive element not set");
    if (which == GATEAU_VEC_TB_A || which == GATEAU_VEC_TB_B) {
        if (!p->kelvin) return fail(GATEAU_ESTATE, "brightness-temperature output not enabled");
        if (p->dirty || p->tb_a.size() != static_cast<size_t>(p->n_ch))
            return fail(GATEAU_ESTATE, "the skydip runs when the plan is prepared (gateau_plan_prepare)");
        src = which == GATEAU_VEC_TB_A ? &p->tb_a : &p->tb_b;
    } else if (needs_tables) {
        if (!p->has_cascade || !p->has_disp) return fail(GATEAU_ESTATE, "cascade and dispersive element must be set");
        // Host-only rebuild (no device upload) so the tables are available without a GPU.
        std::vector<PrimStage> prim;
        std::string err;
        if (!expand_stages(p->stages, p->nu, prim, err)) return fail(GATEAU_EINVAL, "%s", err.c_str());
        const gateau_plan_desc& d = p->desc;
        std::vector<double> c0, c1, c2;
        collapse_cascade(p->nu, prim, d.T_atm_K, d.T_cmb_K, d.eta_taper, d.rho_surf_m, d.eta_pol, c0, c1, c2);
        if (which == GATEAU_VEC_C0) tmp = c0;
        else if (which == GATEAU_VEC_C1) tmp = c1;
        else if (which == GATEAU_VEC_C2) tmp = c2;
        else {
            if (p->pink_auto && p->dirty && which != GATEAU_VEC_PINK_A)
                return fail(GATEAU_ESTATE, "the automatic pink level is set when the plan is prepared");
            const int np = pink_pole_count(d.pink_f_min_hz, d.f_sample_hz);
            std::vector<double> a(static_cast<size_t>(p->n_ch) * np), r(a.size()), dd(p->n_ch);
            for (int c = 0; c < p->n_ch; ++c)
                pink_design_channel(p->has_pink ? p->pink_alpha[c] : 1.0, p->has_pink ? p->pink_A[c] : 0.0,
                                    d.pink_f_min_hz, d.f_sample_hz, np, &a[static_cast<size_t>(c) * np],
                                    &r[static_cast<size_t>(c) * np], &dd[c]);
            if (which == GATEAU_VEC_PINK_A) tmp = a;
            else if (which == GATEAU_VEC_PINK_R) tmp = r;
            else if (which == GATEAU_VEC_PINK_D) tmp = dd;
            else return fail(GATEAU_EINVAL, "unknown vector id %d", which);
        }
        src = &tmp;
    } else if (which == GATEAU_VEC_NU) {
        src = &p->nu;
    } else if (which == GATEAU_VEC_WEIGHT) {
        src = &p->w;
    } else if (which == GATEAU_VEC_ETA_FILT) {
        src = &p->eta_filt;
    } else {
        return fail(GATEAU_EINVAL, "unknown vector id %d", which);
    }
    if (count < src->size()) return fail(GATEAU_EINVAL, "out holds %zu doubles, table has %zu", count, src->size());
    std::copy(src->begin(), src->end(), out);
    return GATEAU_OK;
}

gateau_status gateau_plan_get_state(gateau_plan* p, long long* next_t0, double* pink_state) {
    if (!p) return fail(GATEAU_EINVAL, "plan is NULL");
    if (next_t0) *next_t0 = p->next_t0;
    if (pink_state) {
        if (!p->has_disp) return fail(GATEAU_ESTATE, "dispersive element not set");
        const size_t n = static_cast<size_t>(p->desc.n_pix) * p->n_ch * pink_pole_count(p->desc.pink_f_min_hz, p->desc.f_sample_hz);
        if (!p->d_state.p || p->d_state.bytes < n * sizeof(float)) {
            std::fill(pink_state, pink_state + n, 0.0);
            return GATEAU_OK;
        }
        GATEAU_CUDA(cudaStreamSynchronize(p->last_stream));
        std::vector<float> h(n);
        GATEAU_CUDA(cudaMemcpy(h.data(), p->d_state.p, n * sizeof(float), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) pink_state[i] = h[i];
    }
    return GATEAU_OK;
}

gateau_status gateau_plan_set_state(gateau_plan* p, long long next_t0, const double* pink_state) {
    if (!p || next_t0 < 0) return fail(GATEAU_EINVAL, "plan must be non-NULL and next_t0 >= 0");
    if (pink_state) {
        if (!p->has_disp) return fail(GATEAU_ESTATE, "dispersive element not set");
        gateau_status st = ensure_base(p);
        if (st != GATEAU_OK) return st;
        st = finalize(p);
        if (st != GATEAU_OK) return st;
        const size_t n = static_cast<size_t>(p->desc.n_pix) * p->n_ch * p->n_pole;
        std::vector<float> h(n);
        for (size_t i = 0; i < n; ++i) h[i] = static_cast<float>(pink_state[i]);
        GATEAU_CUDA(cudaStreamSynchronize(p->last_stream));
        GATEAU_CUDA(cudaMemcpy(p->d_state.p, h.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    }
    p->next_t0 = next_t0;
    return GATEAU_OK;
}

gateau_status gateau_plan_set_tiles(gateau_plan* p, int n_groups, int ring_b) {
    if (!p) return fail(GATEAU_EINVAL, "plan is NULL");
    if (ring_b != 0 && (ring_b < 2 || ring_b > kMaxRingB)) return fail(GATEAU_EINVAL, "ring_b must be 0 or 2..%d", kMaxRingB);
    if (n_groups < 0) return fail(GATEAU_EINVAL, "n_groups must be >= 0");
    if (n_groups > 0 && p->has_disp) {
        const int n_ch = p->n_ch;
        if (n_groups > n_ch || ((n_ch + n_groups - 1) / n_groups + 15) / 16 * 16 > 176)
            return fail(GATEAU_EINVAL, "%d channels do not split into %d groups of 1..176", n_ch, n_groups);
    }
    p->tile_groups = n_groups;
    p->tile_ring_b = ring_b;
    p->tune_ms = 0.0;
    p->ref_dirty = true;
    return GATEAU_OK;
}

gateau_status gateau_plan_autotune(gateau_plan* p, long long nt_sample, void* stream, gateau_tile_choice* out) {
    if (!p) return fail(GATEAU_EINVAL, "plan is NULL");
    if (p->desc.precision != GATEAU_PREC_BF16X3) return fail(GATEAU_EINVAL, "only split-BF16 plans have fused tiles");
    if (nt_sample < 1) return fail(GATEAU_EINVAL, "nt_sample must be >= 1");
    gateau_status st = check_complete(p);
    if (st != GATEAU_OK) return st;
    st = ensure_base(p);
    if (st != GATEAU_OK) return st;
    if (p->scan_kind == GATEAU_SCAN_CUSTOM) nt_sample = std::min(nt_sample, p->n_custom);
    nt_sample = std::min(nt_sample, (1LL << 31) / p->desc.n_pix);
    const int n_ch = p->n_ch;
    const int key = (n_ch + 15) / 16;
    gateau_tile_choice res{};
    bool cached = false;
    std::pair<int, int> choice;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);   // held for the lookup only: plans build in parallel
        auto f = g_tune_cache.find(key);
        if (f != g_tune_cache.end()) {
            cached = true;
            choice = f->second;
        }
    }
    if (cached) {
        p->tile_groups = choice.first;
        p->tile_ring_b = choice.second;
        p->ref_dirty = true;
        st = finalize(p);
        if (st != GATEAU_OK) return st;
        res.n_groups = p->fused.n_groups;
        res.n_half = p->fused.n_half;
        res.ring_b = fused_ring_depths(p->fused.n_half, p->fused.ring_b, &res.ring_a);
        if (out) *out = res;
        return GATEAU_OK;
    }
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    const bool timing = p->timing;
    p->timing = false;
    struct Restore {                    // the plan's timing flag, whatever happens below
        gateau_plan* p;
        bool t;
        ~Restore() { p->timing = t; }
    } restore{p, timing};
    const size_t out_bytes = static_cast<size_t>(nt_sample) * p->desc.n_pix * n_ch * sizeof(float);
    GATEAU_CUDA(grow(p, p->d_tune, out_bytes));
    p->tile_groups = 0;
    p->tile_ring_b = 0;
    p->ref_dirty = true;
    st = run_rows(p, 0, nt_sample, cs, false);          // rows of the sample: the same for every tile choice
    if (st != GATEAU_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GATEAU_CUDA(cudaEventCreate(&e0));
    GATEAU_CUDA(cudaEventCreate(&e1));
    struct Events {
        cudaEvent_t a, b;
        ~Events() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } evs{e0, e1};
    const int g0 = (n_ch + 175) / 176;
    std::vector<int> groups{g0, g0 + 1};
    if (g0 != 2 && g0 + 1 != 2) groups.push_back(2);
    double best_ms = 1e300, default_ms = 0.0;
    int best_g = g0, best_rb = kDefaultRingB, n_timed = 0;
    for (int g : groups) {
        if (g > n_ch || ((n_ch + g - 1) / g + 15) / 16 * 16 > 176) continue;
        const int n_half = ((n_ch + g - 1) / g + 15) / 16 * 16;
        for (int rb = 2; rb <= kMaxRingB; ++rb) {
            if (fused_ring_depths(n_half, rb, nullptr) != rb) continue;   // that depth does not fit
            p->tile_groups = g;
            p->tile_ring_b = rb;
            p->ref_dirty = true;
            st = finalize(p);
            if (st != GATEAU_OK) return st;
            const FusedRunDesc r = fused_run(p, 0, nt_sample, p->d_tune.as<float>());
            GATEAU_CUDA(launch_fused_runs(&r, 1, p->n_sm, cs));           // warm-up
            GATEAU_CUDA(cudaEventRecord(e0, cs));
            for (int rep = 0; rep < 2; ++rep) GATEAU_CUDA(launch_fused_runs(&r, 1, p->n_sm, cs));
            GATEAU_CUDA(cudaEventRecord(e1, cs));
            GATEAU_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            GATEAU_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            const double per = ms / 2.0;
            ++n_timed;
            if (g == g0 && rb == kDefaultRingB) default_ms = per;
            if (per < best_ms) {
                best_ms = per;
                best_g = g;
                best_rb = rb;
            }
        }
    }
    p->tile_groups = best_g;
    p->tile_ring_b = best_rb;
    p->ref_dirty = true;
    st = finalize(p);
    if (st != GATEAU_OK) return st;
    p->tune_ms = best_ms;
    p->d_tune.release(p->mo);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = std::make_pair(best_g, best_rb);
    }
    res.n_groups = p->fused.n_groups;
    res.n_half = p->fused.n_half;
    res.ring_b = fused_ring_depths(p->fused.n_half, p->fused.ring_b, &res.ring_a);
    res.ms = best_ms;
    res.default_ms = default_ms;
    res.candidates = n_timed;
    if (out) *out = res;
    return GATEAU_OK;
}

gateau_status gateau_plan_set_wait_budget(gateau_plan* p, long long cycles) {
    if (!p) return fail(GATEAU_EINVAL, "plan is NULL");
    if (cycles < 0) return fail(GATEAU_EINVAL, "the wait budget must be >= 0 cycles");
    p->fused.wait_cycles = cycles;
    return GATEAU_OK;
}

gateau_status gateau_plan_set_timing(gateau_plan* p, int enable) {
    if (!p) return fail(GATEAU_EINVAL, "plan is NULL");
    p->timing = enable != 0;
    return GATEAU_OK;
}

gateau_status gateau_plan_get_timing(gateau_plan* p, double* ms, long long* runs, long long* launches) {
    if (!p) return fail(GATEAU_EINVAL, "plan is NULL");
    if (ms)
        for (int ph = 0; ph < GATEAU_PHASE_COUNT; ++ph) ms[ph] = 0.0;
    if (!p->timed.empty()) GATEAU_CUDA(cudaStreamSynchronize(p->last_stream));
    for (gateau_plan::TimedRun& t : p->timed)
        for (int ph = 0; ph < GATEAU_PHASE_COUNT; ++ph)
            if (t.used[ph]) {
                float e = 0.f;
                GATEAU_CUDA(cudaEventElapsedTime(&e, t.ev[ph][0], t.ev[ph][1]));
                if (ms) ms[ph] += e;
                p->ev_pool.push_back(t.ev[ph][0]);
                p->ev_pool.push_back(t.ev[ph][1]);
            }
    p->timed.clear();
    if (runs) *runs = p->runs;
    if (launches) *launches = p->launches;
    p->runs = 0;
    p->launches = 0;
    return GATEAU_OK;
}

gateau_status gateau_hex_offsets(int R_hex, double spacing_rad, double* out, int count, int* n_out) {
    if (R_hex < 0 || R_hex > 64) return fail(GATEAU_EINVAL, "need 0 <= R_hex <= 64");
    const int n = 1 + 3 * R_hex * (R_hex + 1);
    if (n_out) *n_out = n;
    if (!out || count < n) return fail(GATEAU_EINVAL, "out must hold %d offset pairs", n);
    std::vector<double> v;
    hex_offsets(R_hex, spacing_rad, v);
    std::copy(v.begin(), v.end(), out);
    return GATEAU_OK;
}

}  // extern "C"
