// Internal declarations shared by the host plan code and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gateau.h"
#include "plan_host.h"

namespace gateau {

constexpr int kMaxPoles = 24;          // pink-filter poles supported by the kernels
constexpr int kMaxScanParams = 8;

// Per-row quantities produced by the row-setup kernel and read by the spectral
// producers (32 bytes, one row = one (time sample, spaxel) pair).
struct __align__(16) RowParams {
    float csc;        // 1 / sin(elevation)                                   (Eq. 10)
    int tau_j;        // opacity-table row below the row's PWV
    float tau_f;      // fractional position between rows tau_j and tau_j+1
    int src_idx;      // element offset of cube texel (ia, ie), or -1 outside (Sect. 2.4)
    float src_fa;     // fractional azimuth cell position
    float src_fe;     // fractional elevation cell position
    float pwv;        // line-of-sight PWV (mm), kept for diagnostics
    int src_cell;     // ia * 65536 + ie of the cube cell, or -1 outside
};

// Per-tile summary written by the row setup for the fused kernel: the range of
// opacity-table rows and the cube texel box that the tile's 128 rows touch, so
// that both can be staged in shared memory by tensor copies.
constexpr int kTileRows = 128;
constexpr int kTauBoxRows = 8;                // opacity rows per staged box
constexpr int kTauBoxRowsS = 2;               // opacity rows of the small box (a tile spanning one or two rows)
constexpr int kCubeBoxAz = 12, kCubeBoxEl = 4; // cube texels per staged box (a 128-sample tile of a 30"/s raster spans ~8 x 2 cells)
constexpr int kCubeBoxElS = 2;                 // elevation rows of the small box (a tile whose rows stay in one cell row)
enum { TILE_TAU_FITS = 1, TILE_CUBE_FITS = 2, TILE_HAS_SOURCE = 4, TILE_CUBE_SMALL = 8, TILE_TAU_SMALL = 16 };
struct __align__(16) TileInfo {
    int j0;           // lowest opacity row of the tile
    int ia0, ie0;     // lowest cube cell of the tile's source rows
    int flags;        // TILE_* bits
};

// Everything the kernels read, by value (device pointers + scalars).
struct DevTables {
    // geometry and scan (Sect. 2.4)
    int n_pix;
    const double* pix_off;             // [n_pix][2]
    const double* pix_trig;            // [n_pix][4]: tan dphi, tan dth, sin dth, cos dth
    const float* pix_trig_f;           // the same in float
    double f_sample, h_column, wind;
    int scan_kind;
    double sp[kMaxScanParams];
    double phi0, theta0;
    const double* custom;              // [n_custom][2] or null
    long long n_custom;
    // screen [ny][nx] PWV mm
    const float* screen;
    int nx, ny;
    double pitch;
    // opacity table [n_pwv][2][Kp]: row 2j = tau_j(nu), row 2j+1 = tau_{j+1} - tau_j
    const float* tau;
    int n_pwv;
    double pwv_min, dpwv;
    // source cube [n_az][n_el][Kp], pre-multiplied by c2(nu)/k_B: the source term of the
    // collapsed cascade in kelvin (the caller's cube is kept unscaled beside it)
    const float* cube;
    int n_az, n_el;
    double az0, daz, el0, del;
    // spectral axis
    int n_freq, Kp;
    const float* c0;                   // [Kp] kelvin
    const float* c1;                   // [Kp] kelvin
    const float* c2;                   // [Kp] kelvin per (W/Hz), folded into cube
    // Reference spectrum X_ref = c0 + c1 (1 - e_ref) (source-free, mean PWV, base elevation): the
    // contractions run on D = X - X_ref = c_ref - c1 e + e P'_src
    const float* cref;                 // [Kp] c1 e_ref, kelvin
    const float* ref_pk;               // [n_ch_pad] k_B 1e9 sum H X_ref (W), added to P_KID
    const float* ref_n;                // [n_ch_pad] sum G X_ref + Q X_ref^2, added to N
    // contraction operands, fp32 [n_ch_pad][Kp] (plain path), on D
    int n_ch, n_ch_pad;
    const float* H;                    // eta_filt * w_GHz
    const float* G;                    // H * gamma (nu_GHz + beta) + 2 Q X_ref
    const float* Q;                    // eta_filt^2 * w_GHz
    // epilogue scales: P_KID = kb1e9 * S1 + ref_pk,  sigma = kB * sqrt(noise_scale * (N + ref_n))
    float kb1e9;
    float kB;
    float noise_scale;                 // 1e9 * f_sample
    uint32_t key0, key1;               // Philox key
    int noise_flags;
    // pink noise
    int n_pole;
    const float* pink_a;               // [n_ch][n_pole]
    const float* pink_r;               // [n_ch][n_pole] gain folded in
    const float* pink_d;               // [n_ch] gain folded in
    // brightness-temperature output (Sect. 2.7): out = tb_a[ch] P_tot + tb_b[ch] (K), or null for W.
    // The pink residues and direct term are already multiplied by tb_a.  Both arrays start on
    // 16-byte boundaries (padded to a multiple of 16 channels), so quads of channels load as float4.
    const float* tb_a;
    const float* tb_b;
    unsigned int* status;
};

// Device buffers for the split-BF16 fused path.
struct FusedOperands {
    const uint16_t* B;                 // pre-tiled bf16 operand stages (see kernels_fused.cu)
    int n_half;                        // channels per CTA (multiple of 16)
    int n_groups;                      // channel groups (CTAs per row tile)
    int n_kstage;                      // K stages of fused_kstage() points
    size_t stage_elems;                // bf16 elements per (group, kstage) block
    int tma_inputs;                    // 1: opacity rows and cube texels are staged by tensor copies
    const float* c_tiled;              // [Kp/16][2][16] c_ref and c1 per stage (kelvin)
    long long wait_cycles;             // budget of each pipeline wait (clock64 cycles); drains keep their own
    int ring_b;                        // deepest B ring (filter-operand stages) to use, 2..kMaxRingB
};

constexpr long long kDefaultWaitCycles = 4000000000LL;   // ~2 s at 2 GHz
constexpr int kDefaultRingB = 4;       // B-ring depth the fused kernel takes unless tuned
constexpr int kMaxRingB = 6;

// Opaque 128-byte tensor-map descriptors (CUtensorMap) for the staged inputs.
struct __align__(64) TensorMapBytes {
    unsigned char b[128];
};

// ---- kernel launchers (each enqueues on `stream`, returns cudaGetLastError) ----
cudaError_t launch_row_setup(const DevTables& T, long long t0, long long nt, RowParams* rows,
                             TileInfo* tiles, cudaStream_t stream);
cudaError_t launch_tau_interleave(const float* rows, int n_pwv, int nf, int Kp, float* out, cudaStream_t stream);
cudaError_t launch_scale_cube(const float* raw, const float* c2, long long n_texels, int Kp, float* out,
                              cudaStream_t stream);
cudaError_t launch_psd_fp32(const DevTables& T, const RowParams* rows, long long r0, long long nrows,
                            float* X, cudaStream_t stream);
cudaError_t launch_contract_fp32(const DevTables& T, const float* X, long long r0, long long nrows,
                                 long long t0, long long nt, float* out, cudaStream_t stream);
// One plan's run for a fused launch (several when a server batches its requests' chunks).
struct FusedRunDesc {
    DevTables T;
    FusedOperands F;
    TensorMapBytes tm_tau, tm_tau_s, tm_cube, tm_cube_s;   // the full boxes and the small ones
    const RowParams* rows;
    const TileInfo* tiles;
    long long t0, nt;
    float* out;
};
// One persistent launch over the work items of 1..fused_max_jobs() runs of one launch mode (all
// with two channel groups, or none with two).
cudaError_t launch_fused_runs(const FusedRunDesc* runs, int n, int n_sm, cudaStream_t stream);
int fused_max_jobs();
// B-ring depth (return) and A-ring depth (*nsa) the fused kernel takes for n_half and ring_b.
int fused_ring_depths(int n_half, int ring_b, int* nsa);
// Encodes the tensor maps of the opacity table [n_pwv][Kp] and the cube [n_az][n_el][Kp] (its
// full and small boxes; driver entry point looked up at run time); false if the driver cannot.
bool fused_encode_input_maps(const float* tau, int n_pwv, const float* cube, int n_az, int n_el, int Kp,
                             TensorMapBytes* tm_tau, TensorMapBytes* tm_tau_s, TensorMapBytes* tm_cube,
                             TensorMapBytes* tm_cube_s,
                             std::string& err);
size_t fused_smem_bytes();
int fused_kstage();
// The contraction operands of channel c at point k (k < n_freq; zero past it), in device units (w in
// GHz, X in kelvin): H = eta w, G = H gamma (nu_GHz + beta), Q = eta^2 w (Sect. 2.5 Eq. 16, Sect. 2.6
// Eq. 17), and G' = G + 2 Q X_ref for the reference-spectrum difference.
struct FilterOperands {
    const double* eta = nullptr;      // [n_ch][nf] filter transmission
    const double* w = nullptr;        // [nf] trapezoid weights (Hz)
    const double* nu = nullptr;       // [nf] frequencies (Hz)
    const double* xref = nullptr;     // [nf] reference spectrum (kelvin), for G'
    int nf = 0;
    double gamma = 0, beta = 0;
    void at(int c, int k, double& h, double& g, double& q) const {
        const double e = eta[static_cast<size_t>(c) * nf + k];
        const double wg = w[k] * 1e-9;
        h = e * wg;
        g = h * gamma * (nu[k] * 1e-9 + beta);
        q = e * e * wg;
    }
    double gprime(double g, double q, int k) const { return g + 2.0 * q * xref[k]; }
};
void fused_tile_operands(const FilterOperands& f, int n_ch, int Kp, int n_half, int n_groups,
                         std::vector<uint16_t>& out, size_t& stage_elems);

// Pink noise: chunked linear-recurrence scan adding into out.
struct PinkWork {
    float* agg;                        // [C][S][n_pole]
    int C;                             // chunks per sequence
    long long L;                       // samples per chunk (multiple of 4)
};
void pink_choose_chunks(long long nt, long long S, int& C, long long& L);
// Skydip (Sect. 2.7): for each channel, P_KID and the band-averaged sky brightness temperature at
// n_dip zenith PWVs pwv_lo .. pwv_hi at elevation el (csc_el = 1 / sin el), no source, and the
// least-squares line T_b = a P + b.  hw [n_ch][n_freq] = eta_filt w (Hz), c01 [2][n_freq] = the
// collapsed cascade's c0, c1 (W/Hz), tau the plan's opacity table.  Writes ab [2][n_ch] (FP64:
// a then b) and ab_f (the same in FP32, b at ab_f + ab_f_stride).  2 <= n_dip <= kMaxSkydip.
constexpr int kMaxSkydip = 64;
cudaError_t launch_skydip_fit(const double* hw, const double* c01, const float* tau, int n_freq, int Kp, int n_pwv,
                              double pwv_min, double dpwv, double csc_el, double T_atm, double pwv_lo, double pwv_hi,
                              int n_dip, int n_ch, double* ab, float* ab_f, int ab_f_stride, cudaStream_t stream);

// Exact pink noise (Timmer & Koenig, Sect. 2.6): tk_length(N) = 2^ceil(log2 N) (>= 2);
// launch_tk_realise writes tk [n_total][n_pix][n_ch] (W, times scale[ch] when scale is not null)
// from the per-channel PSD A [n_ch] (W^2/Hz at 1 Hz) and alpha [n_ch], key (k0, k1), using the
// scratch buffers work0, work1 of (n_pix ceil(n_ch/2)) x tk_length(n_total) float2 each;
// launch_tk_add adds tk[0 .. count) into out.
long long tk_length(long long n_total);
// Batched complex FFT of `rows` contiguous rows of length M (a power of two) from a, with b as the
// second buffer (both are overwritten); sign +1: sum e^{+2 pi i jk/M} (unscaled inverse), -1:
// forward.  *result points at whichever of a, b holds the transform.
cudaError_t launch_fft_rows(float2* a, float2* b, long long rows, int M, int sign, const float2** result,
                            cudaStream_t stream);
cudaError_t launch_tk_realise(const double* A, const double* alpha, double f_sample, uint32_t k0, uint32_t k1, int n_pix,
                              int n_ch, long long n_total, const float* scale, float2* work0, float2* work1, float* tk,
                              cudaStream_t stream);
cudaError_t launch_tk_add(float* out, const float* tk, long long count, cudaStream_t stream);

// Common-mode reduction (Sect. 4.3, Eqs. 25-26): sum of rows[0 .. n).pwv into *sum (atomic, FP64);
// log of each channel's band transmission at zenith PWV pwv; T*_a of a TOD tb [nt][n_pix][n_ch]
// (out may be tb) given the run's rows (csc), log_eta_z [n_ch], off_source [n_pix] (S_j) and N_out.
cudaError_t launch_sum_pwv(const RowParams* rows, long long n, double* sum, cudaStream_t stream);
cudaError_t launch_band_transmission(const double* hw, const float* tau, int n_freq, int Kp, int n_pwv, double pwv_min,
                                     double dpwv, double pwv, int n_ch, float* log_eta_z, cudaStream_t stream);
cudaError_t launch_common_mode(const float* tb, float* out, const RowParams* rows, long long nt, int n_pix, int n_ch,
                               const float* log_eta_z, const unsigned char* off_source, int n_out,
                               cudaStream_t stream);

// Preprocessing (Sect. 2.2, Eqs. 1-3), kernels_prep.cu.  Planes are complex [B][n0][n1] with n0, n1
// powers of two.  fft2_planes: 2-D transform in place in a (b scratch).  launch_beam_planes: the far
// field F of B frequencies nu[0..B) (device FP64) on an na x ne offset grid into F, peak-normalised
// (normalise) or with its peak in peak[b] only.
// launch_convolve_source_batch: Eq. 1 for frequencies f0 .. f0+B-1 of the cube I [n_az][n_el][n_freq]
// into P (same layout), with scratch planes K, S, work of B (2 n_az)(2 n_el) each and peak [B].
// launch_smooth_screen: the screen [ny][nx] smoothed by the normalised footprint, scratch planes of
// nx ny each and one device double.
cudaError_t fft2_planes(float2* a, float2* b, int B, int n0, int n1, int sign, cudaStream_t stream);
cudaError_t launch_real_part(const float2* in, float* out, long long n, cudaStream_t stream);
cudaError_t launch_beam_planes(const double* nu, int B, int na, int ne, double d_az, double d_el, double R,
                               double t_edge_db, float2* F, float2* work, float* peak, cudaStream_t stream,
                               bool normalise = true);
cudaError_t launch_convolve_source_batch(const float* I, float* P, const double* nu, int B, int f0, int n_freq,
                                         int n_az, int n_el, double el0, double d_az, double d_el, double R,
                                         double t_edge_db, float2* K, float2* S, float2* work, float* peak,
                                         cudaStream_t stream);
cudaError_t launch_smooth_screen(const float* screen, float* out, int nx, int ny, double pitch, double R,
                                 double t_edge_db, float2* K, float2* S, float2* work, double* sum,
                                 cudaStream_t stream);

cudaError_t launch_pink(const DevTables& T, float* state, const PinkWork& W, long long t0, long long nt,
                        float* out, cudaStream_t stream);

// Host helpers
void set_last_error(const std::string& msg);
uint16_t f32_to_bf16_rn(float x);
float bf16_to_f32(uint16_t h);

}  // namespace gateau
