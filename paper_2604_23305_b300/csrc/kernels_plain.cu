// Row setup (per time sample x spaxel) and the plain FP32 path:
//   row_setup     : scan -> pointing -> screen PWV -> opacity row, airmass, source cell  (Sect. 2.4)
//   psd_fp32      : P_nu[row][nu] after the cascade, materialised in HBM                (Sect. 2.5)
//   contract_fp32 : SIMT contraction against eta_filt (Eq. 16) and the NEP^2 terms (Eq. 17),
//                   epilogue sigma (Eq. 18) + white noise (Eq. 19) -> out                 (Sect. 2.7)
#include <math.h>

#include "device_common.cuh"

namespace gateau {

__device__ __forceinline__ void scan_pointing(const DevTables& T, long long n, double t, double& phi,
                                              double& th) {
    switch (T.scan_kind) {
        case GATEAU_SCAN_DAISY: {  // Eq. 8
            const double r = T.sp[0], w = T.sp[1], W = T.sp[2];
            phi = r * cos(W * t) * sin(w * t);
            th = r * sin(W * t) * sin(w * t);
            break;
        }
        case GATEAU_SCAN_RASTER: {  // user pattern: boustrophedon in azimuth
            const double half = T.sp[0], speed = T.sp[1], step = T.sp[2];
            const int n_rows = static_cast<int>(T.sp[3]);
            const double T_row = 2.0 * half / speed;
            const double k = floor(t / T_row);
            const double s = t - k * T_row;
            phi = (fmod(k, 2.0) == 0.0) ? (-half + speed * s) : (half - speed * s);
            double row = 0.0;
            if (n_rows > 1) {
                const double m = fmod(k, 2.0 * (n_rows - 1));
                row = (m < n_rows) ? m : 2.0 * (n_rows - 1) - m;
            }
            th = (row - 0.5 * (n_rows - 1)) * step;
            break;
        }
        case GATEAU_SCAN_CUSTOM:
            phi = T.custom[2 * n];
            th = T.custom[2 * n + 1];
            break;
        default:
            phi = 0.0;
            th = 0.0;
    }
}

// Python-style floating modulo for m > 0: the result in [0, m).  With q = floor(a / m)
// the remainder a - q m is exact (one fused multiply-add) whenever q is the true
// quotient; a quotient rounded across an integer is corrected by one step of m.
__device__ __forceinline__ double wrap_mod(double a, double m, double inv_m) {
    const double q = floor(a * inv_m);
    double r = fma(-q, m, a);
    if (r < 0.0) r += m;
    if (r >= m) r -= m;
    return r;
}

// What a row needs from its time sample alone (Sect. 2.4): the time, the scan pointing
// and the trigonometry of it that every spaxel reuses.
struct SampleGeom {
    double t, phs, ths;
    float tan_phs, tan_ths, sin_a, cos_a;                 // a = ths + theta0
};

__device__ __forceinline__ SampleGeom sample_geom(const DevTables& T, long long n) {
    SampleGeom g;
    g.t = static_cast<double>(n) / T.f_sample;
    scan_pointing(T, n, g.t, g.phs, g.ths);
    g.tan_phs = static_cast<float>(tan(g.phs));
    g.tan_ths = static_cast<float>(tan(g.ths));
    double sa, ca;
    sincos(g.ths + T.theta0, &sa, &ca);
    g.sin_a = static_cast<float>(sa);
    g.cos_a = static_cast<float>(ca);
    return g;
}

// Reciprocals of the per-plan divisors, formed once per thread.
struct RowScales {
    double inv_pitch, inv_nx, inv_ny, inv_dpwv, inv_daz, inv_del;
    float h_column;
};

__device__ __forceinline__ RowScales row_scales(const DevTables& T) {
    RowScales k;
    k.inv_pitch = 1.0 / T.pitch;
    k.inv_nx = 1.0 / T.nx;
    k.inv_ny = 1.0 / T.ny;
    k.inv_dpwv = 1.0 / T.dpwv;
    k.inv_daz = 1.0 / T.daz;
    k.inv_del = 1.0 / T.del;
    k.h_column = static_cast<float>(T.h_column);
    return k;
}

// Row (sample n, spaxel i).  The spaxel's offsets enter through the angle-addition
// identities, tan(p + d) = (tan p + tan d) / (1 - tan p tan d) and
// sin(a + d) = sin a cos d + cos a sin d, with tan d, sin d, cos d tabulated per spaxel.
// FP64 where precision is spent: time, wind drift, screen coordinates and wrap, table row and
// source cell; FP32 for the offsets' angle additions (a few tens of metres off the scan line at
// ~1e-7 relative), the bilinear weights and the airmass.
__device__ __forceinline__ RowParams make_row(const DevTables& T, const SampleGeom& g, const RowScales& k, int i) {
    const double dphi = T.pix_off[2 * i], dth = T.pix_off[2 * i + 1];
    const float* tr = T.pix_trig_f + 4 * i;
    const double az = g.phs + T.phi0 + dphi;                 // spaxel pointing (Sect. 2.4)
    const double el = g.ths + T.theta0 + dth;
    // Frozen-flow screen coordinates (Eq. 9) and periodic bilinear PWV.
    const double x = static_cast<double>(k.h_column * ((g.tan_phs + tr[0]) / (1.f - g.tan_phs * tr[0]))) + T.wind * g.t;
    const double y = static_cast<double>(k.h_column * ((g.tan_ths + tr[1]) / (1.f - g.tan_ths * tr[1])));
    double gx = wrap_mod(x * k.inv_pitch + 0.5 * T.nx, static_cast<double>(T.nx), k.inv_nx);
    double gy = wrap_mod(y * k.inv_pitch + 0.5 * T.ny, static_cast<double>(T.ny), k.inv_ny);
    if (!(gx >= 0.0 && gx < T.nx) || !(gy >= 0.0 && gy < T.ny)) {   // non-finite pointing
        atomicOr(T.status, GATEAU_STATUS_BAD_INDEX);
        gx = 0.0;
        gy = 0.0;
    }
    const int ix = static_cast<int>(floor(gx)), iy = static_cast<int>(floor(gy));
    const float fx = static_cast<float>(gx - ix), fy = static_cast<float>(gy - iy);
    const int ix1 = (ix + 1 == T.nx) ? 0 : ix + 1, iy1 = (iy + 1 == T.ny) ? 0 : iy + 1;
    const float s00 = T.screen[static_cast<long long>(iy) * T.nx + ix];
    const float s01 = T.screen[static_cast<long long>(iy) * T.nx + ix1];
    const float s10 = T.screen[static_cast<long long>(iy1) * T.nx + ix];
    const float s11 = T.screen[static_cast<long long>(iy1) * T.nx + ix1];
    const double pwv = (1 - fx) * (1 - fy) * s00 + fx * (1 - fy) * s01 + (1 - fx) * fy * s10 + fx * fy * s11;
    // Opacity-table row (linear in PWV, clamped) and airmass (Eq. 10).
    double u = (pwv - T.pwv_min) * k.inv_dpwv;
    if (!(u >= 0.0 && u <= T.n_pwv - 1)) {                          // also catches NaN
        u = fmin(fmax(u, 0.0), static_cast<double>(T.n_pwv - 1));
        atomicOr(T.status, GATEAU_STATUS_PWV_CLAMPED);
    }
    const int j = min(static_cast<int>(floor(u)), T.n_pwv - 2);
    RowParams rp;
    rp.csc = 1.0f / (g.sin_a * tr[3] + g.cos_a * tr[2]);
    rp.tau_j = j;
    rp.tau_f = static_cast<float>(u - j);
    rp.pwv = static_cast<float>(pwv);
    // Source cell (bilinear, zero outside the grid).
    const double su = (az - T.az0) * k.inv_daz, sv = (el - T.el0) * k.inv_del;
    if (su >= 0.0 && su <= T.n_az - 1 && sv >= 0.0 && sv <= T.n_el - 1) {
        const int ia = min(static_cast<int>(floor(su)), T.n_az - 2);
        const int ie = min(static_cast<int>(floor(sv)), T.n_el - 2);
        rp.src_idx = (ia * T.n_el + ie) * T.Kp;
        rp.src_fa = static_cast<float>(su - ia);
        rp.src_fe = static_cast<float>(sv - ie);
        rp.src_cell = ia * 65536 + ie;
    } else {
        rp.src_idx = -1;
        rp.src_fa = 0.f;
        rp.src_fe = 0.f;
        rp.src_cell = -1;
    }
    return rp;
}

// One block of kTileRows threads per tile of kTileRows consecutive samples; a thread
// forms its sample's geometry once and then the rows of every spaxel, stored
// pixel-major within a run (r = i * nt + (n - t0)), so each spaxel's stores are
// contiguous across the block.  With a tile buffer, the block also reduces, per
// spaxel, the tile's opacity-row range and cube box (warp reductions, then the four
// warps' partial results through a shared-memory buffer that alternates on every
// spaxel step, so one barrier per step orders each buffer's writes and its read).
__global__ void __launch_bounds__(kTileRows) row_setup_kernel(DevTables T, long long t0, long long nt,
                                                              RowParams* rows, TileInfo* tiles) {
    constexpr int kWarps = kTileRows / 32;
    __shared__ int s_part[2][kWarps][7];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long tpp = (nt + kTileRows - 1) / kTileRows;
    const RowScales k = row_scales(T);
    int use = 0;                                       // alternates the buffer on every spaxel step
    for (long long b = blockIdx.x; b < tpp; b += gridDim.x) {
        const long long r = b * kTileRows + threadIdx.x;
        const bool valid = r < nt;
        SampleGeom g{};
        if (valid) g = sample_geom(T, t0 + r);
        for (int i = 0; i < T.n_pix; ++i) {
            int jmin = 0x7fffffff, jmax = -1, amin = 0x7fffffff, amax = -1, emin = 0x7fffffff, emax = -1, has = 0;
            if (valid) {
                const RowParams rp = make_row(T, g, k, i);
                rows[static_cast<long long>(i) * nt + r] = rp;
                jmin = jmax = rp.tau_j;
                if (rp.src_cell >= 0) {
                    amin = amax = rp.src_cell >> 16;
                    emin = emax = rp.src_cell & 0xffff;
                    has = 1;
                }
            }
            if (!tiles) continue;
            const unsigned full = 0xffffffffu;
            jmin = __reduce_min_sync(full, jmin);
            jmax = __reduce_max_sync(full, jmax);
            amin = __reduce_min_sync(full, amin);
            amax = __reduce_max_sync(full, amax);
            emin = __reduce_min_sync(full, emin);
            emax = __reduce_max_sync(full, emax);
            has = __reduce_add_sync(full, has);
            const int buf = use;
            use ^= 1;
            int* part = s_part[buf][warp];
            if (lane == 0) {
                part[0] = jmin; part[1] = jmax; part[2] = amin; part[3] = amax;
                part[4] = emin; part[5] = emax; part[6] = has;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int v[7] = {0x7fffffff, -1, 0x7fffffff, -1, 0x7fffffff, -1, 0};
                for (int w = 0; w < kWarps; ++w) {
                    const int* q = s_part[buf][w];
                    v[0] = min(v[0], q[0]); v[1] = max(v[1], q[1]);
                    v[2] = min(v[2], q[2]); v[3] = max(v[3], q[3]);
                    v[4] = min(v[4], q[4]); v[5] = max(v[5], q[5]);
                    v[6] += q[6];
                }
                TileInfo ti;
                ti.j0 = v[0];
                ti.ia0 = v[6] ? v[2] : 0;
                ti.ie0 = v[6] ? v[4] : 0;
                int f = 0;
                if (v[1] - v[0] <= kTauBoxRows - 1) f |= TILE_TAU_FITS;
                if (v[1] - v[0] <= kTauBoxRowsS - 1) f |= TILE_TAU_SMALL;
                if (v[6]) {
                    f |= TILE_HAS_SOURCE;
                    if (v[3] + 1 - v[2] <= kCubeBoxAz - 1 && v[5] + 1 - v[4] <= kCubeBoxEl - 1) f |= TILE_CUBE_FITS;
                    if (v[5] + 1 - v[4] <= kCubeBoxElS - 1) f |= TILE_CUBE_SMALL;   // every row in one cell row
                }
                ti.flags = f;
                tiles[static_cast<long long>(i) * tpp + b] = ti;
            }
        }
    }
}

cudaError_t launch_row_setup(const DevTables& T, long long t0, long long nt, RowParams* rows, TileInfo* tiles,
                             cudaStream_t stream) {
    const long long tpp = (nt + kTileRows - 1) / kTileRows;        // one block per time tile
    long long grid = tpp < 148LL * 16 ? tpp : 148LL * 16;
    row_setup_kernel<<<static_cast<unsigned>(grid), kTileRows, 0, stream>>>(T, t0, nt, rows, tiles);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Spectral power after the cascade, FP32 (Sect. 2.5), using the exact collapse
// P = c0 + c1 (1 - eta_atm) + c2 eta_atm P_src with eta_atm = exp(-csc tau_z), written as its
// difference from the plan's source-free reference spectrum X_ref = c0 + c1 (1 - e_ref):
// D = c1 e_ref - c1 eta_atm + eta_atm c2 P_src (the contraction adds back the reference's
// integrals).  One block per row, 4 consecutive frequencies per thread.
// ---------------------------------------------------------------------------
__global__ void psd_fp32_kernel(DevTables T, const RowParams* __restrict__ rows, long long r0,
                                float* __restrict__ X) {
    const long long row = blockIdx.x;
    const RowParams rp = rows[r0 + row];
    const float* tA = T.tau + static_cast<long long>(2 * rp.tau_j) * T.Kp;   // tau_j
    const float* tD = tA + T.Kp;                                             // tau_{j+1} - tau_j
    const bool has_src = rp.src_idx >= 0;
    const float fa = rp.src_fa, fe = rp.src_fe;
    const float w00 = (1.f - fa) * (1.f - fe), w10 = fa * (1.f - fe), w01 = (1.f - fa) * fe, w11 = fa * fe;
    const float* s00 = T.cube + (has_src ? rp.src_idx : 0);
    const float* s10 = s00 + static_cast<long long>(T.n_el) * T.Kp;
    const float* s01 = s00 + T.Kp;
    const float* s11 = s10 + T.Kp;
    float* xr = X + row * T.Kp;
    for (int k = threadIdx.x * 4; k < T.Kp; k += blockDim.x * 4) {
        const float4 a4 = *reinterpret_cast<const float4*>(tA + k);
        const float4 d4 = *reinterpret_cast<const float4*>(tD + k);
        const float4 cr4 = *reinterpret_cast<const float4*>(T.cref + k);
        const float4 c14 = *reinterpret_cast<const float4*>(T.c1 + k);
        float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
        if (has_src) {
            const float4 q00 = *reinterpret_cast<const float4*>(s00 + k);
            const float4 q10 = *reinterpret_cast<const float4*>(s10 + k);
            const float4 q01 = *reinterpret_cast<const float4*>(s01 + k);
            const float4 q11 = *reinterpret_cast<const float4*>(s11 + k);
            p.x = w00 * q00.x + w10 * q10.x + w01 * q01.x + w11 * q11.x;
            p.y = w00 * q00.y + w10 * q10.y + w01 * q01.y + w11 * q11.y;
            p.z = w00 * q00.z + w10 * q10.z + w01 * q01.z + w11 * q11.z;
            p.w = w00 * q00.w + w10 * q10.w + w01 * q01.w + w11 * q11.w;
        }
        float4 o;
#define GATEAU_PSD(c)                                                  \
    {                                                                  \
        const float tau = fmaf(rp.tau_f, d4.c, a4.c);                  \
        const float e = expf(-rp.csc * tau);                           \
        o.c = fmaf(e, p.c, fmaf(-c14.c, e, cr4.c));                    \
    }
        GATEAU_PSD(x) GATEAU_PSD(y) GATEAU_PSD(z) GATEAU_PSD(w)
#undef GATEAU_PSD
        *reinterpret_cast<float4*>(xr + k) = o;
    }
}

// cube[t][k] = raw[t][k] * c2[k]: the source term of the collapsed cascade in kelvin.
__global__ void scale_cube_kernel(const float4* __restrict__ raw, const float4* __restrict__ c2, long long n4,
                                  int Kp4, float4* __restrict__ out) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n4;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float4 a = raw[i], c = c2[i % Kp4];
        out[i] = make_float4(a.x * c.x, a.y * c.y, a.z * c.z, a.w * c.w);
    }
}

cudaError_t launch_scale_cube(const float* raw, const float* c2, long long n_texels, int Kp, float* out,
                              cudaStream_t stream) {
    const long long n4 = n_texels * Kp / 4;
    long long grid = (n4 + 255) / 256;
    if (grid > 148LL * 16) grid = 148LL * 16;
    scale_cube_kernel<<<static_cast<unsigned>(grid), 256, 0, stream>>>(
        reinterpret_cast<const float4*>(raw), reinterpret_cast<const float4*>(c2), n4, Kp / 4,
        reinterpret_cast<float4*>(out));
    return cudaGetLastError();
}

// The opacity table as the kernels read it, [n_pwv][2][Kp]: row 2j holds tau_j, row 2j+1
// tau_{j+1} - tau_j (float difference; 0 for the last j), zero past n_freq.  One block per output row.
__global__ void tau_interleave_kernel(const float* __restrict__ rows, int n_pwv, int nf, int Kp, float* __restrict__ out) {
    const int r = blockIdx.x, j = r >> 1;
    const float* a = rows + static_cast<size_t>(j) * nf;
    float* o = out + static_cast<size_t>(r) * Kp;
    for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
        float v = 0.f;
        if (k < nf) v = (r & 1) ? (j + 1 < n_pwv ? a[nf + k] - a[k] : 0.f) : a[k];
        o[k] = v;
    }
}

cudaError_t launch_tau_interleave(const float* rows, int n_pwv, int nf, int Kp, float* out, cudaStream_t stream) {
    if (n_pwv <= 0) return cudaSuccess;
    tau_interleave_kernel<<<static_cast<unsigned>(2 * n_pwv), 256, 0, stream>>>(rows, n_pwv, nf, Kp, out);
    return cudaGetLastError();
}

cudaError_t launch_psd_fp32(const DevTables& T, const RowParams* rows, long long r0, long long nrows,
                            float* X, cudaStream_t stream) {
    if (nrows <= 0) return cudaSuccess;
    psd_fp32_kernel<<<static_cast<unsigned>(nrows), 256, 0, stream>>>(T, rows, r0, X);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP32 SIMT contraction of D = X - X_ref.  For a block of 128 rows x 64 channels:
//   S1[r][ch] = sum_k D[r][k] H[ch][k]                      (Eq. 16, kelvin*GHz, less the reference's)
//   N [r][ch] = sum_k D[r][k] G[ch][k] + D[r][k]^2 Q[ch][k]  (Eq. 17 without 2 kB^2 1e9, less the
//               reference's; G carries the cross term 2 Q X_ref)
// 256 threads, each 8 rows x 4 consecutive channels, K in steps of 16 with a
// register-prefetched shared-memory tile.
// ---------------------------------------------------------------------------
constexpr int kBM = 128, kBN = 64, kBK = 16;

__global__ __launch_bounds__(256) void contract_fp32_kernel(DevTables T, const float* __restrict__ X,
                                                            long long r0, long long nrows, long long t0,
                                                            long long nt, float* __restrict__ out) {
    __shared__ __align__(16) float Xs[kBK][kBM + 4];
    __shared__ __align__(16) float Hs[kBK][kBN];
    __shared__ __align__(16) float Gs[kBK][kBN];
    __shared__ __align__(16) float Qs[kBK][kBN];

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const long long rb = static_cast<long long>(blockIdx.x) * kBM;   // row block within the chunk
    const int cb = blockIdx.y * kBN;                                  // channel block
    const int Kp = T.Kp;

    // global -> register loaders
    const int xa_row0 = tid >> 2, xa_kq = tid & 3;                    // 2 float4 of X per thread
    const int hb_ch = tid >> 2, hb_kq = tid & 3;                      // 1 float4 of H, G, Q each
    float4 xr[2], hr, gr, qr;
    auto load_tiles = [&](int k0) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const long long row = rb + xa_row0 + 64 * u;
            xr[u] = (row < nrows) ? *reinterpret_cast<const float4*>(X + row * Kp + k0 + 4 * xa_kq)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const long long hoff = static_cast<long long>(cb + hb_ch) * Kp + k0 + 4 * hb_kq;
        hr = *reinterpret_cast<const float4*>(T.H + hoff);
        gr = *reinterpret_cast<const float4*>(T.G + hoff);
        qr = *reinterpret_cast<const float4*>(T.Q + hoff);
    };
    auto store_tiles = [&]() {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int row = xa_row0 + 64 * u;
            Xs[4 * xa_kq + 0][row] = xr[u].x;
            Xs[4 * xa_kq + 1][row] = xr[u].y;
            Xs[4 * xa_kq + 2][row] = xr[u].z;
            Xs[4 * xa_kq + 3][row] = xr[u].w;
        }
        Hs[4 * hb_kq + 0][hb_ch] = hr.x; Hs[4 * hb_kq + 1][hb_ch] = hr.y;
        Hs[4 * hb_kq + 2][hb_ch] = hr.z; Hs[4 * hb_kq + 3][hb_ch] = hr.w;
        Gs[4 * hb_kq + 0][hb_ch] = gr.x; Gs[4 * hb_kq + 1][hb_ch] = gr.y;
        Gs[4 * hb_kq + 2][hb_ch] = gr.z; Gs[4 * hb_kq + 3][hb_ch] = gr.w;
        Qs[4 * hb_kq + 0][hb_ch] = qr.x; Qs[4 * hb_kq + 1][hb_ch] = qr.y;
        Qs[4 * hb_kq + 2][hb_ch] = qr.z; Qs[4 * hb_kq + 3][hb_ch] = qr.w;
    };

    float s1[8][4], sn[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) s1[i][j] = sn[i][j] = 0.f;

    load_tiles(0);
    for (int k0 = 0; k0 < Kp; k0 += kBK) {
        __syncthreads();
        store_tiles();
        __syncthreads();
        if (k0 + kBK < Kp) load_tiles(k0 + kBK);
#pragma unroll
        for (int k = 0; k < kBK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&Xs[k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&Xs[k][ty * 8 + 4]);
            const float4 h = *reinterpret_cast<const float4*>(&Hs[k][tx * 4]);
            const float4 g = *reinterpret_cast<const float4*>(&Gs[k][tx * 4]);
            const float4 q = *reinterpret_cast<const float4*>(&Qs[k][tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float hv[4] = {h.x, h.y, h.z, h.w};
            const float gv[4] = {g.x, g.y, g.z, g.w};
            const float qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float x2 = a[i] * a[i];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    s1[i][j] = fmaf(a[i], hv[j], s1[i][j]);
                    sn[i][j] = fmaf(a[i], gv[j], fmaf(x2, qv[j], sn[i][j]));
                }
            }
        }
    }

    // Epilogue: P_KID (Eq. 16), sigma (Eqs. 17-18), white noise (Eq. 19).
    const int ch0 = cb + tx * 4;
    const bool white = (T.noise_flags & GATEAU_NOISE_WHITE) != 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const long long row = rb + ty * 8 + i;
        if (row >= nrows) continue;
        const long long rg = r0 + row;
        const int pix = static_cast<int>(rg / nt);
        const long long n = t0 + (rg - static_cast<long long>(pix) * nt);
        float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        if (white) z = white_normals4(n, pix, ch0 >> 2, T.key0, T.key1);
        float* orow = out + ((n - t0) * T.n_pix + pix) * static_cast<long long>(T.n_ch);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int ch = ch0 + j;
            if (ch < T.n_ch) {
                const float pk = fmaf(T.kb1e9, s1[i][j], T.ref_pk[ch]);
                const float sigma = T.kB * sqrtf(T.noise_scale * fmaxf(sn[i][j] + T.ref_n[ch], 0.f));
                const float v = fmaf(sigma, f4_get(z, j), pk);
                orow[ch] = T.tb_a ? fmaf(T.tb_a[ch], v, T.tb_b[ch]) : v;   // K (Sect. 2.7) or W
            }
        }
    }
}

cudaError_t launch_contract_fp32(const DevTables& T, const float* X, long long r0, long long nrows,
                                 long long t0, long long nt, float* out, cudaStream_t stream) {
    if (nrows <= 0) return cudaSuccess;
    dim3 grid(static_cast<unsigned>((nrows + kBM - 1) / kBM), static_cast<unsigned>(T.n_ch_pad / kBN));
    contract_fp32_kernel<<<grid, 256, 0, stream>>>(T, X, r0, nrows, t0, nt, out);
    return cudaGetLastError();
}

}  // namespace gateau
