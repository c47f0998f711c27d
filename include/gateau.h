/*
 * gateau.h -- C ABI of the B300 time-ordered-data simulator (hot path of
 * gateau, arXiv 2604.23305).
 *
 * For every time sample n and IFU spaxel i the library computes, on one GPU:
 *   screen PWV (Sect. 2.4, Eq. 9) -> zenith opacity and airmass (Eq. 10)
 *   -> source sample (Sect. 2.4) -> radiative-transfer cascade (Sect. 2.5,
 *   Eqs. 11-15) -> dispersive element (Sect. 2.3, Eqs. 6-7; Sect. 2.5, Eq. 16)
 *   -> photon noise (Sect. 2.6, Eqs. 17-19) + pink noise (Sect. 2.6, Eq. 20)
 *   -> out[n - t0][i][ch] = P_KID + P_wn + P_pn in W (Sect. 2.7, Eq. 21).
 *
 * Conventions shared by every entry point
 *   - Pointers are plain host or device addresses; no library types cross the
 *     boundary except the opaque plan.  "host" pointers are read during the
 *     call only; "device" pointers must be valid CUDA device memory of the
 *     plan's device.  Setters COPY their inputs into plan-owned memory: the
 *     caller may free or reuse its buffers when the setter returns.
 *   - Arrays are C-contiguous, row-major, in the shapes given below.
 *   - Angles are radians, frequencies Hz, temperatures K, lengths m, PWV mm,
 *     spectral power W/Hz, output power W.
 *   - Every call returns a gateau_status; on failure a thread-local message is
 *     available from gateau_last_error().  Argument errors are detected on the
 *     host before anything is enqueued.  No entry point traps or aborts.
 *   - A plan is used by one host thread at a time.
 */
#ifndef GATEAU_H
#define GATEAU_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GATEAU_ABI_VERSION 1

typedef struct gateau_plan gateau_plan;

typedef enum {
    GATEAU_OK = 0,
    GATEAU_EINVAL = -1,       /* an argument is out of range or inconsistent        */
    GATEAU_ENOMEM = -2,       /* host or device allocation failed                    */
    GATEAU_ECUDA = -3,        /* a CUDA runtime call failed (message has the name)   */
    GATEAU_EORDER = -4,       /* t0 neither 0 nor the end of the previous chunk      */
    GATEAU_ESTATE = -5,       /* a required setter has not been called               */
    GATEAU_EDEVICE = -6,      /* the device status word reports an error bit         */
    GATEAU_ETIMEOUT = -7,     /* a bounded device-side wait ran out                  */
    GATEAU_EUNSUPPORTED = -8  /* the device cannot run the requested path            */
} gateau_status;

/* Contraction precision of the dispersive-element integral (Sect. 2.5, Eq. 16). */
enum {
    GATEAU_PREC_FP32 = 0,     /* FP32 spectra, FP32 SIMT contraction                 */
    GATEAU_PREC_BF16X3 = 1    /* fused kernel: FP32 spectra split into BF16 hi+lo,
                                 3 tcgen05 products (hi*hi + hi*lo + lo*hi) with FP32
                                 accumulation for P_KID; 1 BF16 product per noise term */
};

/* Where a setter's array lives. */
enum { GATEAU_MEM_HOST = 0, GATEAU_MEM_DEVICE = 1 };

/* Scan patterns (Sect. 2.4).  params:
 *   STARE  : none                                   phi = theta = 0
 *   DAISY  : r_petal, omega, Omega (Eq. 8)          phi = r cos(Omega t) sin(omega t),
 *                                                   theta = r sin(Omega t) sin(omega t)
 *   RASTER : half_width, speed, row_step, n_rows    boustrophedon rows in azimuth of
 *            period 2 half_width/speed, row k running +phi (even k) or -phi (odd k),
 *            elevation walking the n_rows positions up and down, centred on 0
 *   CUSTOM : none; a [n_custom][2] table of (phi, theta) indexed by the sample number */
enum { GATEAU_SCAN_STARE = 0, GATEAU_SCAN_DAISY = 1, GATEAU_SCAN_RASTER = 2, GATEAU_SCAN_CUSTOM = 3 };

/* Dispersive elements (Sect. 2.3). */
enum {
    GATEAU_DISP_FILTERBANK = 0,   /* Eq. 7: channels fed in series, highest f first          */
    GATEAU_DISP_LORENTZIAN = 1,   /* Eq. 6: independent Lorentzians (grating)                */
    GATEAU_DISP_CUSTOM = 2        /* user eta_filt[ch][nu] (measured filters, multichroic)   */
};

/* Cascade stage kinds (Sect. 2.5). */
enum {
    GATEAU_STAGE_REFLECTIVE = 0,  /* Eq. 12 with eta (scalar or per frequency)               */
    GATEAU_STAGE_OHMIC = 1,       /* Eq. 12 with eta = 1 - eps_ref sqrt(nu/nu_ref) (Eq. 13)  */
    GATEAU_STAGE_REFRACTIVE = 2   /* Eq. 15, Eq. 14, Eq. 15 (three primitive stages), or Eq. 14
                                     alone when anti-reflection coated                        */
};

/* A stage temperature equal to GATEAU_T_SKY couples the stage to the sky: its
 * emission is (1 - eta_atm) B(T_atm) + eta_atm B(T_cmb) for the same spaxel and
 * time (Sect. 2.5, secondary spillover). */
#define GATEAU_T_SKY (-1.0)

/* Noise switches (plan-wide).  Bit set = component added. */
enum { GATEAU_NOISE_WHITE = 1, GATEAU_NOISE_PINK = 2 };

/* Device status bits read by gateau_plan_status(). */
enum {
    GATEAU_STATUS_PWV_CLAMPED = 1u,    /* informational: a PWV left the table range (clamped)   */
    GATEAU_STATUS_WAIT_TIMEOUT = 2u,   /* error: a pipeline wait in the fused kernel ran out     */
    GATEAU_STATUS_BAD_INDEX = 4u       /* error: an index check failed and the access was skipped */
};

/* Plan description (everything fixed for a simulation). */
typedef struct {
    int n_freq;                    /* spectral points, >= 2                                     */
    double f_lo_hz, f_hi_hz;       /* uniform grid, both end points included                    */
    double f_sample_hz;            /* readout rate; sample n is at t = n / f_sample (Eq. 18)   */
    int n_pix;                     /* spaxels, >= 1                                             */
    const double* pix_offsets_rad; /* host [n_pix][2] (dphi_i, dtheta_i) (Sect. 2.3)           */
    double T_atm_K;                /* atmosphere temperature (Sect. 2.4)                        */
    double T_cmb_K;                /* CMB temperature, 2.725 in the paper (Sect. 2.5, Eq. 11)  */
    double h_column_m;             /* PWV column height (Eq. 9)                                 */
    double wind_mps;               /* frozen-flow wind along +x (Eq. 9)                        */
    double eta_taper;              /* taper efficiency (Sect. 2.3)                              */
    double rho_surf_m;             /* rms surface roughness for the Ruze factor (Eq. 5)        */
    double eta_pol;                /* polarisation efficiency (Eq. 11)                          */
    double delta_al_J;             /* superconducting gap (Sect. 2.3); 2 Delta/h is the cutoff */
    double eta_pb;                 /* pair-breaking efficiency (Sect. 2.3, Eq. 17)             */
    unsigned long long seed;       /* Philox4x32-10 key for all noise draws                     */
    int precision;                 /* GATEAU_PREC_*                                             */
    int noise_flags;               /* GATEAU_NOISE_* bits                                       */
    double pink_f_min_hz;          /* lowest pole of the pink-noise filter, e.g. 1/T_scan      */
} gateau_plan_desc;

/* One cascade stage, after the atmosphere (stage 0 is always the atmosphere). */
typedef struct {
    int kind;                      /* GATEAU_STAGE_*                                            */
    double T_K;                    /* physical temperature, or GATEAU_T_SKY                     */
    double eta;                    /* REFLECTIVE: efficiency when eta_nu is NULL                */
    const double* eta_nu;          /* REFLECTIVE: host [n_freq] efficiencies, or NULL           */
    double eps_ref, nu_ref_hz;     /* OHMIC: reference emissivity at nu_ref                    */
    double d_m, n_index, tan_delta;/* REFRACTIVE: thickness, refractive index, loss tangent    */
    double T_refl_K;               /* REFRACTIVE: temperature seen by the two surface passes   */
    int ar_coated;                 /* REFRACTIVE: nonzero drops the surface passes              */
} gateau_stage;

/* Sizes of a finished plan. */
typedef struct {
    int n_freq, n_freq_padded;     /* spectral points and the padded contraction depth          */
    int n_ch, n_pix, n_pole;       /* channels, spaxels, pink-filter poles                      */
    long long next_t0;             /* first sample of the next chunk                            */
    size_t device_bytes;           /* device memory owned by the plan                           */
    int staged_inputs;             /* 1 when the fused kernel stages its gathers by tensor copies
                                      (set by the first BF16X3 run; 0 before it or on fallback)   */
    int tile_groups, tile_half;    /* BF16X3 fused tiles (after prepare): channel groups and the
                                      channels of a group (2 groups: 2-CTA clusters share tiles)  */
    int ring_a, ring_b;            /* pipeline depths the fused kernel takes: spectrum-row stages
                                      and filter-operand stages in shared memory                   */
    double tune_ms;                /* gateau_plan_autotune: the chosen tiles' time on the tuning
                                      sample (ms; 0 when not measured by this plan)               */
} gateau_plan_info;

/* Host-built FP64 tables, for inspection and tests (gateau_plan_get_vector). */
enum {
    GATEAU_VEC_NU = 0,             /* [n_freq] grid (Hz)                                        */
    GATEAU_VEC_WEIGHT = 1,         /* [n_freq] trapezoid weights (Hz)                           */
    GATEAU_VEC_ETA_FILT = 2,       /* [n_ch][n_freq] eta_filt (Eqs. 6-7, cutoff applied)        */
    GATEAU_VEC_C0 = 3,             /* [n_freq] cascade constant term (W/Hz), see gateau_set_cascade */
    GATEAU_VEC_C1 = 4,             /* [n_freq] coefficient of (1 - eta_atm) (W/Hz)              */
    GATEAU_VEC_C2 = 5,             /* [n_freq] coefficient of eta_atm * P_src                   */
    GATEAU_VEC_PINK_A = 6,         /* [n_ch][n_pole] discrete poles a_j                         */
    GATEAU_VEC_PINK_R = 7,         /* [n_ch][n_pole] residues r_j (gain folded in)              */
    GATEAU_VEC_PINK_D = 8,         /* [n_ch] direct term d (gain folded in)                     */
    GATEAU_VEC_TB_A = 9,           /* [n_ch] skydip scale a (K/W), see gateau_set_output_kelvin  */
    GATEAU_VEC_TB_B = 10           /* [n_ch] skydip offset b (K)                                */
};

/* Library version string and the calling thread's last error message. */
const char* gateau_version(void);
const char* gateau_last_error(void);

/* Number of CUDA devices visible (0 on a machine without a GPU; never fails). */
int gateau_device_count(void);

/* Create a plan from desc (copied).  Builds the frequency grid on the host;
 * allocates no device memory yet.  EINVAL on inconsistent sizes.  *out is set
 * to NULL on failure. */
gateau_status gateau_plan_create(const gateau_plan_desc* desc, gateau_plan** out);

/* Free every host and device resource of the plan (NULL is a no-op).  The
 * caller must have synchronised any stream the plan ran on. */
void gateau_plan_destroy(gateau_plan* plan);

/* Source cube P_nu,src (Sect. 2.2, after the beam convolution of Eq. 1), W/Hz,
 * cube[n_az][n_el][n_freq] float32 on the grid az = az0 + ia*daz, el = el0 +
 * ie*del (el is absolute elevation).  Bilinear sampling, zero outside the grid
 * (Sect. 2.4).  n_az, n_el >= 2, daz, del > 0.  mem: GATEAU_MEM_HOST/DEVICE. */
gateau_status gateau_set_source_cube(gateau_plan* plan, const float* cube, int n_az, int n_el,
                                     double az0_rad, double daz_rad, double el0_rad, double del_rad,
                                     int mem);

/* PWV screen screen[ny][nx] float32 (mm) on a periodic grid of pitch pitch_m;
 * cell (0,0) sits at x = -nx/2*pitch, y = -ny/2*pitch (Sect. 2.4, Eq. 9).  When
 * is_epl is nonzero the values are extra path length and become
 * PWV = EPL/6.587 + pwv0_mm (Sect. 2.2, Eq. 4).  nx, ny >= 2. */
gateau_status gateau_set_atmosphere_screen(gateau_plan* plan, const float* screen, int nx, int ny,
                                           double pitch_m, int is_epl, double pwv0_mm, int mem);

/* Zenith table table[n_pwv][n_freq] float32 on the PWV grid pwv_min + j*dpwv
 * (Sect. 2.4): opacity tau_z when is_opacity is nonzero, else transmission
 * eta_z (stored as -ln max(eta_z, 1e-30)).  Interpolated linearly in opacity;
 * PWV outside the grid is clamped (status bit GATEAU_STATUS_PWV_CLAMPED).
 * n_pwv >= 2, dpwv > 0. */
gateau_status gateau_set_atmosphere_table(gateau_plan* plan, const float* table, int n_pwv,
                                          double pwv_min_mm, double dpwv_mm, int is_opacity, int mem);

/* Cascade after the atmosphere, in the order the signal meets it (Sect. 2.5,
 * Eqs. 12-15; Tables 1-2).  The library collapses the literal stage-by-stage
 * recurrence into P_nu = c0 + c1 (1 - eta_atm) + c2 eta_atm P_src, an exact
 * identity of Eq. 12 because every stage is affine in P and in eta_atm; c0, c1,
 * c2 are built in FP64 (gateau_plan_get_vector).  0 <= n_stage <= 64. */
gateau_status gateau_set_cascade(gateau_plan* plan, int n_stage, const gateau_stage* stages);

/* Dispersive element (Sect. 2.3, Eqs. 6-7): n_ch channels with centre f_c_hz[ch],
 * resolving power R[ch] and peak efficiency eta_peak[ch] (host arrays), or, for
 * GATEAU_DISP_CUSTOM, custom_eta[n_ch][n_freq] (host FP64) and f_c/R/eta_peak
 * ignored.  Frequencies below 2 Delta_Al / h are zeroed.  1 <= n_ch <= 4096. */
gateau_status gateau_set_dispersive_element(gateau_plan* plan, int kind, int n_ch,
                                            const double* f_c_hz, const double* R,
                                            const double* eta_peak, const double* custom_eta);

/* Pink detector noise (Sect. 2.6, Eq. 20) per channel: one-sided PSD level
 * A[ch] (W^2/Hz at 1 Hz, 0 disables the channel) and slope alpha[ch] in
 * [0, 3] (host arrays [n_ch]).  A = NULL puts every channel's knee at 1 Hz:
 * A[ch] is then the white noise level NEP^2 (Eq. 17, the one-sided white PSD)
 * of the source-free sky at the screen's mean PWV and the scan's base
 * elevation, evaluated in FP64 when the plan is prepared (and again when the
 * screen, table, scan, cascade or dispersive element change).  Realised by a pole-zero filter: poles at
 * f_min 10^(j/3) up to f_sample/2, zeros 10^(alpha/6) above each pole,
 * matched-z, parallel (partial-fraction) form, zero state at sample 0.
 * Requires gateau_set_dispersive_element first (ESTATE otherwise). */
gateau_status gateau_set_pink_noise(gateau_plan* plan, const double* A, const double* alpha);

/* Exact pink noise (Sect. 2.6; Timmer & Koenig 1995) instead of the pole-zero
 * filter, for a scan of n_total samples (0 restores the filter).  When the plan is
 * prepared, the device draws each (spaxel i, channel ch) series whole: Fourier
 * coefficients of a real series of length M = 2^ceil(log2 n_total) with real and
 * imaginary parts N(0, M f_s S(f_j) / 4) at f_j = j f_s / M (0 < j < M/2), a real
 * Nyquist coefficient N(0, M f_s S / 2), no DC term, S(f) = A f^-alpha from
 * gateau_set_pink_noise (one-sided, W^2/Hz at 1 Hz), normals from Philox4x32-10 with
 * counter (j >> 1 lo, j >> 1 hi, i, 2^30 | ch) and Box-Muller pair j & 1; the inverse
 * DFT's first n_total samples are the pink term.  The plan then holds them as a
 * device array [n_total][n_pix][n_ch] float32 (and needs twice n_pix ceil(n_ch/2) M
 * complex64 of scratch while it is prepared); runs add their samples and may not go
 * past n_total (EINVAL).  Used only with GATEAU_NOISE_PINK.  EINVAL unless
 * 0 <= n_total <= 2^30. */
gateau_status gateau_set_pink_timmer_koenig(gateau_plan* plan, long long n_total);

/* Scan pattern (Sect. 2.4, Eq. 8) with scan offset (phi0, theta0).  params has
 * n_params doubles as listed at GATEAU_SCAN_*.  CUSTOM takes custom[n_custom][2]
 * (phi, theta) per sample (host or device per mem); runs may not go past
 * n_custom samples (EINVAL). */
gateau_status gateau_set_scan(gateau_plan* plan, int kind, const double* params, int n_params,
                              double phi0_rad, double theta0_rad, const double* custom,
                              long long n_custom, int mem);

/* Output units (Sect. 2.7).  enable = 0 (the default): detected power P_tot in W.
 * enable != 0: brightness temperature in K by a simulated skydip.  When the plan
 * is prepared, the device sweeps the zenith PWV over n_pwv uniformly spaced
 * values pwv_lo_mm .. pwv_hi_mm (both included) at the scan's base elevation
 * theta0 with no source and no noise, and for every channel records P_KID
 * (Eq. 16) and the band-averaged line-of-sight brightness temperature of the
 * isothermal atmosphere, T_b = T_atm sum eta_filt w (1 - eta_atm) / sum
 * eta_filt w; the least-squares line T_b = a P_KID + b (FP64) then maps every
 * output sample: out = a P_tot + b (gateau_plan_get_vector GATEAU_VEC_TB_A/B
 * after gateau_plan_prepare).  A channel whose power does not change over the
 * sweep gets a = 0.  Needs the table and scan before the plan is prepared.
 * EINVAL unless 0 <= pwv_lo < pwv_hi and 2 <= n_pwv <= 64. */
gateau_status gateau_set_output_kelvin(gateau_plan* plan, int enable, double pwv_lo_mm, double pwv_hi_mm, int n_pwv);

/* Simulate samples n = t0 .. t0+nt-1 for all spaxels into dev_out
 * [nt][n_pix][n_ch] float32 (W, or K with gateau_set_output_kelvin), device memory owned by the caller.  Enqueued
 * on `stream` (a cudaStream_t, NULL = legacy default stream); returns without
 * synchronising.  t0 must be 0 (restarts the pink-noise state) or the end of
 * the previous chunk (EORDER otherwise), so a scan may be produced in chunks
 * of any size with results identical to one call.  The first call after a
 * setter uploads derived tables (synchronous).  Once the plan is prepared and a
 * first run has sized its buffers for chunks of this length, a run enqueues
 * stream work only, so runs can be captured into a CUDA graph and replayed (a
 * replay repeats the captured chunks; the chunk at t0 = 0 resets the pink-filter
 * states within the graph).  ESTATE if the source,
 * screen, table, cascade, dispersive element or scan is missing. */
gateau_status gateau_run(gateau_plan* plan, long long t0, long long nt, float* dev_out, void* stream);

/* Same as gateau_run but writes to host memory host_out[nt][n_pix][n_ch];
 * the library simulates in chunks on `stream` and copies each chunk back
 * while the next one runs.  Synchronous: returns when host_out is complete.
 * Page-locked host_out gives the full copy bandwidth. */
gateau_status gateau_run_host(gateau_plan* plan, long long t0, long long nt, float* host_out,
                              void* stream);

/* Synchronise the plan's last stream and read (and clear) the device status
 * word into *flags (GATEAU_STATUS_* bits).  Returns EDEVICE when an error bit
 * (anything but GATEAU_STATUS_PWV_CLAMPED) is set, ETIMEOUT for WAIT_TIMEOUT. */
gateau_status gateau_plan_status(gateau_plan* plan, unsigned int* flags);

/* Sizes and device memory of the plan (after all setters). */
gateau_status gateau_plan_get_info(gateau_plan* plan, gateau_plan_info* info);

/* Copy a host-built FP64 table (GATEAU_VEC_*) into out, which holds `count`
 * doubles; EINVAL when count is smaller than the table. */
gateau_status gateau_plan_get_vector(gateau_plan* plan, int which, double* out, size_t count);

/* Checkpoint / resume of the chunked simulation: the next sample index and the
 * pink-filter states pink_state[n_pix][n_ch][n_pole] (FP64 host; may be NULL in
 * get).  Synchronises the plan's last stream. */
gateau_status gateau_plan_get_state(gateau_plan* plan, long long* next_t0, double* pink_state);
gateau_status gateau_plan_set_state(gateau_plan* plan, long long next_t0, const double* pink_state);

/* Tile shapes of the fused split-BF16 kernel.  A tile is 128 consecutive samples of
 * one spaxel (one TMEM lane per sample) x a group of channels, built and contracted
 * in stages of 16 spectral points (one K = 16 MMA step), so the rows and the spectral
 * stage are fixed by the tensor-core shapes; what a plan chooses is the channel
 * split and the pipeline depth.  n_groups: channel groups of at most 176 channels
 * (>= ceil(n_ch / 176), and n_ch / n_groups >= 1; 0 restores the default, the fewest
 * groups); exactly 2 groups run as 2-CTA clusters that build every spectrum row once
 * and share it, any other count as independent CTAs.  ring_b: the deepest ring of
 * filter-operand stages to take, 2..6 (0: the default 4), as far as shared memory
 * leaves room for at least as many spectrum-row stages.  Takes effect at the next
 * prepare or run; results are the same for every choice (within the split-BF16
 * tolerance; bit-identical output is not promised across choices).  EINVAL
 * outside those ranges. */
gateau_status gateau_plan_set_tiles(gateau_plan* plan, int n_groups, int ring_b);

/* Tile autotuner (project-written): for a BF16X3 plan with all setters done, time
 * every candidate (channel groups: the fewest, one more, and 2 when that is not
 * already a candidate; B-ring depths 2..6 that fit) on the first nt_sample samples
 * of the scan (CUDA events on `stream`, one warm-up and two timed launches of the
 * fused kernel each, into device scratch owned by the plan and freed afterwards),
 * keep the fastest, and cache it for the process under the plan's shape class (its
 * channel count in 16-channel blocks, which fixes every candidate's group width and
 * ring depths).  A later plan of a cached class
 * takes the cached choice without measuring.  The run state of the plan (next
 * sample, pink-filter states) is not touched.  *out (may be NULL) receives the
 * chosen n_groups, ring_b, its time and how many candidates were timed (0: from the
 * cache).  Synchronous.  EINVAL for a FP32 plan or nt_sample < 1. */
typedef struct {
    int n_groups, n_half, ring_b, ring_a;
    double ms;                     /* the chosen tiles' time per launch on the sample (ms)      */
    double default_ms;             /* the default tiles' time on the same sample (ms; 0 if cached) */
    int candidates;                /* configurations timed (0: taken from the cache)            */
} gateau_tile_choice;
gateau_status gateau_plan_autotune(gateau_plan* plan, long long nt_sample, void* stream, gateau_tile_choice* out);

/* Budget of each pipeline wait of the fused split-BF16 kernel, in SM clock cycles
 * (clock64; default 4e9, about 2 s at 2 GHz).  A wait that runs out sets
 * GATEAU_STATUS_WAIT_TIMEOUT in the plan's status word, every role of the kernel
 * stops, the kernel waits (with the default budget, whatever this one is) for its
 * own copies and tensor-core operations in flight, frees its tensor memory and
 * returns, so the CUDA context stays usable and gateau_plan_status reports
 * ETIMEOUT.  The output of that run is incomplete.  A budget far below a
 * pipeline stage's latency (0, say) makes a run time out on purpose, which is how
 * the time-out path is tested; it affects later runs of this plan only.  The
 * bounded waits are the kernel's guard against a pipeline that stops making
 * progress (Sect. 2.5-2.6 give no counterpart).  EINVAL for a negative budget. */
gateau_status gateau_plan_set_wait_budget(gateau_plan* plan, long long cycles);

/* Phase timing.  With timing enabled, every run records CUDA events on its
 * stream around each phase; gateau_plan_get_timing synchronises the plan's last
 * stream, adds the elapsed milliseconds per phase since the previous call into
 * ms[GATEAU_PHASE_COUNT] (which it zeroes first), reports the runs and kernel
 * launches counted in that interval, and restarts the interval.  Launches are
 * counted whether or not timing is enabled. */
enum {
    GATEAU_PHASE_ROWS = 0,         /* per-row scan, pointing, PWV, airmass, source cell      */
    GATEAU_PHASE_SPECTRUM = 1,     /* FP32 path only: spectra materialised in HBM            */
    GATEAU_PHASE_CONTRACT = 2,     /* contraction + photon noise (fused kernel for BF16X3)   */
    GATEAU_PHASE_PINK = 3,         /* pink-noise scan                                        */
    GATEAU_PHASE_COUNT = 4
};
gateau_status gateau_plan_set_timing(gateau_plan* plan, int enable);
gateau_status gateau_plan_get_timing(gateau_plan* plan, double* ms, long long* runs, long long* launches);

/* Packed-hexagon spaxel layout (Sect. 2.3): circumradius R_hex spaxels (0..64),
 * spacing spacing_rad; writes 1 + 3 R (R+1) (dphi, dtheta) pairs into
 * out[count][2] (host) in rings from the centre.  Returns EINVAL if count is
 * too small; *n_out receives the spaxel count. */
gateau_status gateau_hex_offsets(int R_hex, double spacing_rad, double* out, int count, int* n_out);

/* Build everything a plan derives from its setters' inputs -- the collapsed
 * cascade, the filter operands, the pink-noise filters -- and upload it, so
 * that the first gateau_run only enqueues work.  Optional: gateau_run does it
 * when needed.  ESTATE if a setter is missing.  Blocks the calling thread
 * (host work and synchronous uploads); plans of different threads are
 * independent, so a service can prepare plans on worker threads. */
gateau_status gateau_plan_prepare(gateau_plan* plan);

/* ---- Preprocessing (Sect. 2.2, Eqs. 1-3), on the device ---------------------
 * The telescope far field F from a Gaussian aperture illumination whose amplitude
 * falls to t_edge_db (dB, e.g. -10) at the rim of radius R_tel_m,
 * A(r) = 10^((t_edge/20)(r/R)^2) for r < R, 0 outside (Eq. 2), as
 * F = |2-D DFT of A|^2 normalised to a peak of 1 (Eq. 3).  A is sampled in
 * wavelengths on spacings 1/(n d) so that F lands on the angular grid of pitch d:
 * gateau_beam_far_field writes dev_F[n_freq][n_a][n_e] (float32, device) with the
 * offset (q d_az, p d_el) at index (q mod n_a, p mod n_e).
 * gateau_convolve_source evaluates Eq. 1 on a specific-intensity cube
 * dev_I[n_az][n_el][n_freq] (W m^-2 Hz^-1 sr^-1, float32, device; cell (a, e) at
 * az0 + a d_az, el0 + e d_el): dev_P = A_p sum over cells of I cos(el') F(dphi,
 * dtheta) d_az d_el (W/Hz, the layout of gateau_set_source_cube), A_p = pi R^2,
 * the beam taken on the offset grid of twice the cube (a linear convolution).
 * gateau_smooth_screen convolves a periodic screen dev_screen[ny][nx] (pitch_m)
 * with the footprint A(r), r in metres, normalised to unit sum (line-of-sight PWV).
 * Sizes n_a, n_e, n_az, n_el, nx, ny: powers of two.  nu_hz: host [n_freq] (Hz).
 * Enqueued on `stream` with scratch from its stream-ordered pool; the beam and
 * convolution calls synchronise the stream before returning.  EINVAL on bad sizes,
 * pitches or pointers (dev_P may not alias dev_I). */
gateau_status gateau_beam_far_field(const double* nu_hz, int n_freq, int n_a, int n_e, double d_az_rad, double d_el_rad,
                                    double R_tel_m, double t_edge_db, float* dev_F, void* stream);
gateau_status gateau_convolve_source(const float* dev_I, int n_az, int n_el, int n_freq, const double* nu_hz,
                                     double el0_rad, double d_az_rad, double d_el_rad, double R_tel_m, double t_edge_db,
                                     float* dev_P, void* stream);
gateau_status gateau_smooth_screen(const float* dev_screen, int nx, int ny, double pitch_m, double R_tel_m,
                                   double t_edge_db, float* dev_out, void* stream);

/* ---- Downstream: common-mode reduction (Sect. 4.3, Eqs. 25-26) ----------
 * gateau_mean_zenith_pwv: the zenith PWV averaged over the observation, i.e. the
 * mean of the line-of-sight screen PWV over every row (n, i) with n < n_total,
 * computed on the device (rows by the row-setup kernel, FP64 sum); synchronous.
 * gateau_common_mode: for a brightness-temperature TOD tb[nt][n_pix][n_ch]
 * (device, K, samples t0 .. t0+nt-1, e.g. from a run after
 * gateau_set_output_kelvin), writes out[nt][n_pix][n_ch] (device; may be tb)
 *   T*_a,i = T_b,i / eta_i - (1 - eta_i) / (eta_i N_out) sum_j S_j T_b,j / (1 - eta_j)
 * with S_j = 1 for spaxels farther than r_out_rad from the IFU centre (N_out of
 * them, at least one or EINVAL), eta_i = eta_z^csc(el_i(t)) at spaxel i's own
 * elevation (Eq. 10), and eta_z of a channel the zenith transmission at
 * pwv_mean_mm averaged over the band with the channel's weights eta_filt w.
 * Enqueued on `stream`; uses the plan's row buffer, so it must not overlap a run
 * of the same plan. */
gateau_status gateau_mean_zenith_pwv(gateau_plan* plan, long long n_total, double* pwv_mean_mm);
gateau_status gateau_common_mode(gateau_plan* plan, long long t0, long long nt, const float* tb, float* out,
                                 double pwv_mean_mm, double r_out_rad, void* stream);

/* Several plans' chunks on one stream, the way a server batches the time chunks
 * of its admitted requests.  plans[k] runs samples t0s[k] .. t0s[k]+nts[k]-1
 * into outs[k] (device) exactly as gateau_run would, with the same chunk-order
 * rules and bit-identical results.  The split-BF16 contractions of all the
 * batch's plans share persistent launches of the fused kernel -- one launch for
 * the plans with two channel groups (177-352 channels: 2-CTA clusters) and one
 * for the others, each over every work item (time tile x spaxel x channel
 * group) of up to 28 plans -- so uneven requests fill the GPU together; the
 * row setup and the noise phases stay per plan.  FP32 plans run one by one.
 * The phase timing of gateau_plan_get_timing reports a shared launch under
 * each of its plans; the launch count counts it once.  0 < n <= 256; the whole
 * batch is validated before anything is enqueued. */
gateau_status gateau_run_batch(gateau_plan* const* plans, const long long* t0s, const long long* nts,
                               float* const* outs, int n, void* stream);

/* Upper bound of the device memory a plan holds (bytes), from the shapes its
 * setters will receive and the longest chunk it will run: desc as for
 * gateau_plan_create, n_ch channels, an n_az x n_el source cube, an nx x ny
 * screen, an n_pwv-row table, chunks of at most chunk_samples samples, and
 * n_custom_pointing custom-scan samples (0 for built-in scans).  Used by
 * servers to admit a request before its plan exists.  Not included: the exact
 * pink-noise realisation (gateau_set_pink_timmer_koenig: n_total n_pix n_ch
 * float32 held, twice n_pix ceil(n_ch/2) 2^ceil(log2 n_total) complex64 while the
 * plan is prepared) and, with brightness-temperature output or the common-mode
 * reduction, n_ch n_freq doubles of eta_filt w (transient for the skydip).
 * EINVAL on bad sizes. */
gateau_status gateau_plan_estimate_bytes(const gateau_plan_desc* desc, int n_ch, int n_az, int n_el, int nx, int ny,
                                         int n_pwv, long long chunk_samples, long long n_custom_pointing,
                                         size_t* bytes);

/* ---- Serving: many simulations sharing one GPU (continuous batching) -----
 * The paper runs one simulation per call (Sect. 3).  A server runs a stream of
 * them -- requests, each a whole simulation (a plan and a scan length) that
 * arrives at some time -- the way a shared simulation service would: it admits
 * a request as soon as one of its max_active slots and enough of its device
 * memory budget are free (first come, first served), creates the request's
 * plan at that moment through the caller's factory, runs the scan in chunks of
 * time samples on one of its streams, copies every chunk's TOD to the host,
 * and destroys the plan (release callback) when the last chunk has arrived,
 * which frees the slot and the memory for the next arrivals.  Requests admitted
 * while others run are on the GPU at the same time: each active request keeps
 * two chunks in flight on its own stream, so their kernels and copies overlap.
 * A request's TOD is bit-identical to gateau_run of the same plan over the
 * same chunks, alone or in any mix. */
typedef struct gateau_server gateau_server;

typedef struct {
    size_t budget_bytes;        /* device memory for admitted requests: their plans (as
                                   requested) plus two chunk buffers each (three with shared
                                   launches) */
    int max_active;             /* requests admitted at once (slots), 1..256 */
    long long chunk_samples;    /* time samples per chunk, >= 1 ... */
    size_t max_chunk_bytes;     /* ... reduced so that one chunk's TOD stays within this many
                                   bytes (>= 4096; also sizes the pinned host staging) */
    int n_streams;              /* CUDA streams, 1..256; admitted request k (in admission
                                   order) runs on stream k mod n_streams */
    int dry_run;                /* 1: scheduling only, no CUDA call and no plan use: a chunk of D
                                   detector samples occupies its stream for
                                   D * dry_seconds_per_sample on a virtual clock (host tests) */
    double dry_seconds_per_sample;
    int n_builders;             /* 0..64 threads that create (factory) and prepare
                                   (gateau_plan_prepare) admitted requests' plans while the
                                   running requests' chunks are launched; 0 builds on the thread
                                   running the server (always so in a dry run) */
    int shared_launches;        /* 0: every request's chunks run on its own stream (their kernels
                                   overlap through the streams).  1: rounds -- the next chunk of
                                   every admitted request with a free chunk buffer -- each run as
                                   one gateau_run_batch on the server's compute stream, so the
                                   requests' split-BF16 contractions share persistent fused
                                   launches; each request's checksum and copy to the host follow
                                   its round on its own stream, which runs at a higher priority
                                   than the compute stream.  A round is formed when none is in
                                   flight, or when one is and every active request can join; each
                                   request has three chunk buffers.  Results are identical. */
} gateau_server_desc;

typedef struct {
    double arrival_s;           /* seconds after gateau_server_run starts; non-decreasing */
    long long nt;               /* scan length in samples, >= 1 */
    int n_pix, n_ch;            /* TOD row shape: the plan's spaxels and channels */
    size_t device_bytes;        /* the plan's device memory (gateau_plan_estimate_bytes) */
    float* host_out;            /* NULL, or host [nt][n_pix][n_ch] that receives the TOD */
} gateau_request;

/* Factory: create the plan of request `request` (index into the array given to
 * gateau_server_run), ready to run from t0 = 0; NULL marks the request failed.
 * With n_builders > 0 it is called on builder threads (several at once, each
 * for a different request); otherwise on the thread running the server.
 * Release: the server is done with the plan (all chunks on the host); the
 * caller destroys it.  Release is called on the thread running the server. */
typedef gateau_plan* (*gateau_plan_factory)(void* user, int request);
typedef void (*gateau_plan_release)(void* user, int request, gateau_plan* plan);

typedef struct {
    int n_requests, n_done, n_failed;
    double p50_latency_s, p99_latency_s;   /* arrival -> last chunk on the host, over done requests
                                              (linear interpolation between order statistics) */
    double mean_latency_s, max_latency_s;
    double makespan_s;                     /* run start -> last completion */
    double detector_samples;               /* sum of nt * n_pix * n_ch over done requests */
    double throughput;                     /* detector_samples / makespan_s */
    size_t peak_bytes;                     /* most budget held at once */
    int peak_active;                       /* most requests admitted at once */
    double overlap;                        /* mean number of requests with chunks in flight,
                                              sampled at every chunk launch */
    long long rounds;                      /* shared launches: rounds run (gateau_run_batch calls) */
    double mean_round;                     /* shared launches: mean requests per round */
} gateau_server_stats;

/* Create / destroy a server.  Create allocates the pinned host staging
 * (2 x max_active x max_chunk_bytes) and the device chunk buffers lazily per
 * admitted request.  EINVAL on out-of-range fields. */
gateau_status gateau_server_create(const gateau_server_desc* desc, gateau_server** out);
void gateau_server_destroy(gateau_server* server);

/* Run requests[0..n-1] to completion in real time (dry_run: virtual time):
 * requests become visible at their arrival_s.  A request whose device_bytes plus
 * chunk buffers exceed the whole budget, or whose plan the factory cannot make,
 * or whose run fails, is marked failed and the others go on.  Returns after the
 * last request finished; stats may be NULL.  ECUDA aborts the run (every admitted
 * plan is released first).  n <= 1000000. */
gateau_status gateau_server_run(gateau_server* server, const gateau_request* requests, int n,
                                gateau_plan_factory create, gateau_plan_release release, void* user,
                                gateau_server_stats* stats);

/* Outcome of request `request` of the last run: state (0 pending, 2 done,
 * 3 failed), latency (arrival -> done, s), admission time (s after the start)
 * and the TOD checksum {sum, sum of squares} (float64, accumulated on the GPU
 * per chunk in a fixed order, so equal TODs give equal checksums). */
gateau_status gateau_server_request_result(gateau_server* server, int request, int* state, double* latency_s,
                                           double* admitted_s, double* checksum2);

/* Allocation-free pink-noise scan.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory while they run
 * (an embedding runtime that owns a fixed memory pool, a real-time loop where
 * cudaMalloc's device synchronisation and unbounded latency are not allowed,
 * or a process whose memory was all reserved at start-up).  It adds the pink
 * noise of samples t0 .. t0+nt-1 into out, exactly like the pink phase of
 * gateau_run, using only buffers the caller passes plus 4 MiB of scratch that
 * the library reserves as a static device array on every GPU that loads it
 * (held until the process exits).  It calls no allocator.
 *   pink_a, pink_r : device [n_ch][n_pole] poles and residues (gain folded in),
 *                    e.g. the GATEAU_VEC_PINK_A / GATEAU_VEC_PINK_R tables as float
 *   pink_d         : device [n_ch] direct terms (GATEAU_VEC_PINK_D as float)
 *   state          : device [n_pix][n_ch][n_pole] filter state before sample t0
 *                    (zeros at the start of a scan), updated in place
 *   out            : device [nt][n_pix][n_ch], the noise is added in place
 *   seed           : the plan seed (Philox key), so the draws match gateau_run
 * Sizes with n_pix * n_ch * n_pole above 1048576 are rejected (EINVAL) before
 * anything is enqueued; longer scans take fewer, longer chunks so that their
 * states fit.  The first call on a device looks up the scratch address
 * (cudaGetSymbolAddress) with that device current.  Under CUDA's default lazy
 * module loading that lookup can load the library's device code on that device,
 * which reserves the array and may synchronise: real-time callers should make
 * one warm-up call at start-up, before their loop and before any stream
 * capture; later calls reserve nothing.  All calls share the scratch and leave their
 * chunk states in it (nothing in it needs to start at zero: every state is
 * written before it is read), so calls whose kernels overlap on the GPU --
 * on different streams, or from different threads -- race; serialise them. */
gateau_status gateau_pink_noise_noalloc(const float* pink_a, const float* pink_r, const float* pink_d,
                                        int n_pix, int n_ch, int n_pole, unsigned long long seed,
                                        long long t0, long long nt, float* state, float* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GATEAU_H */
