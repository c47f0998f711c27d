// Host-side FP64 construction of the plan tables (no CUDA here).
//
//   frequency grid + trapezoid weights          (integrals of Eqs. 16-17)
//   Johnson-Nyquist spectral power              (Sect. 2.5)
//   stage expansion (reflective/Ohmic/refractive) and the cascade collapse
//     P = c0 + c1 (1 - eta_atm) + c2 eta_atm P_src       (Sect. 2.5, Eqs. 11-15)
//   dispersive element eta_filt[ch][nu]          (Sect. 2.3, Eqs. 6-7)
//   pink-noise pole-zero filter in parallel form (Sect. 2.6, Eq. 20)
//   packed-hexagon spaxel offsets               (Sect. 2.3)
#include "plan_host.h"

#include <math.h>

#include <algorithm>
#include <complex>
#include <numeric>

namespace gateau {

std::vector<double> make_grid(int n, double f_lo, double f_hi) {
    std::vector<double> nu(n);
    const double step = (f_hi - f_lo) / (n - 1);
    for (int k = 0; k < n; ++k) nu[k] = f_lo + k * step;
    nu[n - 1] = f_hi;
    return nu;
}

std::vector<double> make_trapezoid(const std::vector<double>& nu) {
    const int n = static_cast<int>(nu.size());
    const double d = (nu[n - 1] - nu[0]) / (n - 1);
    std::vector<double> w(n, d);
    w[0] = w[n - 1] = 0.5 * d;
    return w;
}

double jn_power(double T, double nu) {
    if (!(T > 0.0)) return 0.0;
    const double x = kH * nu / (kKB * T);
    if (x > 700.0) return 0.0;
    return kH * nu / expm1(x);
}

static double ohmic_eta(double eps, double nu_ref, double nu) { return 1.0 - eps * sqrt(nu / nu_ref); }
static double refr_eta(double d, double n, double tand, double nu) {
    return exp(-2.0 * M_PI * d * n * tand * nu / kC);
}
static double refl_eta(double n) {
    const double r = (1.0 - n) / (1.0 + n);
    return 1.0 - r * r;
}

bool expand_stages(const std::vector<StageSpec>& stages, const std::vector<double>& nu,
                   std::vector<PrimStage>& out, std::string& err) {
    out.clear();
    const size_t nf = nu.size();
    for (size_t s = 0; s < stages.size(); ++s) {
        const StageSpec& st = stages[s];
        const bool sky = st.T_K == GATEAU_T_SKY;
        if (!sky && !(st.T_K >= 0.0)) {
            err = "stage " + std::to_string(s) + ": temperature must be >= 0 or GATEAU_T_SKY";
            return false;
        }
        if (st.kind == GATEAU_STAGE_REFLECTIVE) {
            PrimStage p{std::vector<double>(nf), sky, st.T_K};
            for (size_t k = 0; k < nf; ++k) p.eta[k] = st.eta_nu.empty() ? st.eta : st.eta_nu[k];
            out.push_back(std::move(p));
        } else if (st.kind == GATEAU_STAGE_OHMIC) {
            if (!(st.nu_ref_hz > 0.0)) {
                err = "stage " + std::to_string(s) + ": ohmic nu_ref must be > 0";
                return false;
            }
            PrimStage p{std::vector<double>(nf), sky, st.T_K};
            for (size_t k = 0; k < nf; ++k) p.eta[k] = ohmic_eta(st.eps_ref, st.nu_ref_hz, nu[k]);
            out.push_back(std::move(p));
        } else if (st.kind == GATEAU_STAGE_REFRACTIVE) {
            if (!(st.n_index > 0.0) || !(st.d_m >= 0.0) || !(st.tan_delta >= 0.0)) {
                err = "stage " + std::to_string(s) + ": refractive d, n, tan_delta out of range";
                return false;
            }
            PrimStage bulk{std::vector<double>(nf), sky, st.T_K};
            for (size_t k = 0; k < nf; ++k) bulk.eta[k] = refr_eta(st.d_m, st.n_index, st.tan_delta, nu[k]);
            if (st.ar_coated) {
                out.push_back(std::move(bulk));
            } else {
                const bool sky_r = st.T_refl_K == GATEAU_T_SKY;
                PrimStage surf{std::vector<double>(nf, refl_eta(st.n_index)), sky_r, st.T_refl_K};
                out.push_back(surf);
                out.push_back(std::move(bulk));
                out.push_back(surf);
            }
        } else {
            err = "stage " + std::to_string(s) + ": unknown kind";
            return false;
        }
    }
    for (const PrimStage& p : out)
        for (double e : p.eta)
            if (!(e >= 0.0 && e <= 1.0)) {
                err = "a stage efficiency lies outside [0, 1]";
                return false;
            }
    return true;
}

// Collapse of the cascade.  Carry P = alpha + beta e + gamma e P_src through the
// stages, starting from stage 0 (the atmosphere) applied to P_0 (Eq. 11):
//   P_1 = e (a P_src + B_cmb) + (1 - e) B_atm  ->  alpha = B_atm, beta = B_cmb - B_atm, gamma = a
// A stage with emission B_k: alpha <- eta alpha + (1-eta) B_k, beta <- eta beta, gamma <- eta gamma.
// A sky-coupled stage emits B_atm + e (B_cmb - B_atm), adding (1-eta)(B_cmb - B_atm) to beta.
// Finally c0 = alpha + beta, c1 = -beta, c2 = gamma.
void collapse_cascade(const std::vector<double>& nu, const std::vector<PrimStage>& prim, double T_atm,
                      double T_cmb, double eta_taper, double rho_surf, double eta_pol, std::vector<double>& c0,
                      std::vector<double>& c1, std::vector<double>& c2) {
    const size_t nf = nu.size();
    c0.assign(nf, 0.0);
    c1.assign(nf, 0.0);
    c2.assign(nf, 0.0);
    for (size_t k = 0; k < nf; ++k) {
        const double Batm = jn_power(T_atm, nu[k]);
        const double Bcmb = jn_power(T_cmb, nu[k]);
        const double lam = kC / nu[k];
        const double ruze = exp(-pow(4.0 * M_PI * rho_surf / lam, 2));   // Eq. 5 (reading)
        double alpha = Batm, beta = Bcmb - Batm, gamma = eta_taper * ruze * eta_pol;
        for (const PrimStage& p : prim) {
            const double e = p.eta[k];
            if (p.sky) {
                alpha = e * alpha + (1.0 - e) * Batm;
                beta = e * beta + (1.0 - e) * (Bcmb - Batm);
            } else {
                alpha = e * alpha + (1.0 - e) * jn_power(p.T, nu[k]);
                beta = e * beta;
            }
            gamma = e * gamma;
        }
        c0[k] = alpha + beta;
        c1[k] = -beta;
        c2[k] = gamma;
    }
}

bool build_filters(int kind, int n_ch, const double* f_c, const double* R, const double* eta_peak,
                   const double* custom, const std::vector<double>& nu, double delta_al_J,
                   std::vector<double>& eta, std::string& err) {
    const int nf = static_cast<int>(nu.size());
    eta.assign(static_cast<size_t>(n_ch) * nf, 0.0);
    if (kind == GATEAU_DISP_CUSTOM) {
        if (!custom) {
            err = "custom dispersive element needs custom_eta";
            return false;
        }
        std::copy(custom, custom + static_cast<size_t>(n_ch) * nf, eta.begin());
    } else {
        if (!f_c || !R || !eta_peak) {
            err = "dispersive element needs f_c, R and eta_peak";
            return false;
        }
        for (int c = 0; c < n_ch; ++c)
            if (!(f_c[c] > 0.0) || !(R[c] > 0.0)) {
                err = "channel " + std::to_string(c) + ": f_c and R must be > 0";
                return false;
            }
        auto lor = [&](int c, double v) {
            const double x = 2.0 * R[c] * (v / f_c[c] - 1.0);
            return 1.0 / (1.0 + x * x);                                     // Eq. 6 (reading)
        };
        if (kind == GATEAU_DISP_LORENTZIAN) {
            for (int c = 0; c < n_ch; ++c)
                for (int k = 0; k < nf; ++k) eta[static_cast<size_t>(c) * nf + k] = eta_peak[c] * lor(c, nu[k]);
        } else if (kind == GATEAU_DISP_FILTERBANK) {
            // Eq. 7: highest centre frequency first; each numerator loses what the
            // channels upstream (higher f) already took.
            std::vector<int> order(n_ch);
            std::iota(order.begin(), order.end(), 0);
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return f_c[a] > f_c[b]; });
            std::vector<double> taken(nf, 0.0);
            for (int c : order)
                for (int k = 0; k < nf; ++k) {
                    const double v = (eta_peak[c] - taken[k]) * lor(c, nu[k]);
                    eta[static_cast<size_t>(c) * nf + k] = v;
                    taken[k] += v;
                }
        } else {
            err = "unknown dispersive element kind";
            return false;
        }
    }
    const double cutoff = 2.0 * delta_al_J / kH;                            // Sect. 2.3
    for (int c = 0; c < n_ch; ++c)
        for (int k = 0; k < nf; ++k)
            if (nu[k] < cutoff) eta[static_cast<size_t>(c) * nf + k] = 0.0;
    return true;
}

int pink_pole_count(double f_min, double f_sample) {
    return static_cast<int>(floor(3.0 * log10(0.5 * f_sample / f_min) + 1e-9)) + 1;
}

// One channel: poles p_j = f_min 10^(j/3), zeros q_j = p_j 10^(alpha/6), matched z
// (a_j = exp(-2 pi p_j / f_s), b_j likewise), H(w) = prod (1 - b_j w)/(1 - a_j w) =
// d + sum_j r_j / (1 - a_j w); gain g so that (2/f_s) g^2 |H(1 Hz)|^2 = A.
void pink_design_channel(double alpha, double A, double f_min, double f_sample, int n_pole, double* a_out,
                         double* r_out, double* d_out) {
    std::vector<double> a(n_pole), b(n_pole);
    for (int j = 0; j < n_pole; ++j) {
        const double p = f_min * pow(10.0, j / 3.0);
        const double q = p * pow(10.0, alpha / 6.0);
        a[j] = exp(-2.0 * M_PI * p / f_sample);
        b[j] = exp(-2.0 * M_PI * q / f_sample);
    }
    double d = 1.0;
    for (int j = 0; j < n_pole; ++j) d *= b[j] / a[j];
    std::complex<double> H(1.0, 0.0);
    const std::complex<double> zinv = std::polar(1.0, -2.0 * M_PI * 1.0 / f_sample);
    for (int j = 0; j < n_pole; ++j) H *= (1.0 - b[j] * zinv) / (1.0 - a[j] * zinv);
    const double g = A > 0.0 ? sqrt(A * 0.5 * f_sample) / std::abs(H) : 0.0;
    for (int j = 0; j < n_pole; ++j) {
        double num = 1.0, den = 1.0;
        for (int m = 0; m < n_pole; ++m) {
            num *= 1.0 - b[m] / a[j];
            if (m != j) den *= 1.0 - a[m] / a[j];
        }
        a_out[j] = a[j];
        r_out[j] = g * num / den;
    }
    *d_out = g * d;
}

// Packed hexagon: axial coordinates (q, r) with max(|q|, |r|, |q + r|) <= R_hex,
// position (spacing (q + r/2), spacing sqrt(3)/2 r); ordered by ring, then by
// angle atan2 in [0, 2 pi).
int hex_offsets(int R_hex, double spacing, std::vector<double>& out) {
    struct P {
        int ring;
        double ang, x, y;
    };
    std::vector<P> pts;
    for (int q = -R_hex; q <= R_hex; ++q)
        for (int r = -R_hex; r <= R_hex; ++r) {
            const int s = -q - r;
            const int ring = std::max(std::abs(q), std::max(std::abs(r), std::abs(s)));
            if (ring > R_hex) continue;
            const double x = spacing * (q + 0.5 * r), y = spacing * (sqrt(3.0) / 2.0) * r;
            double ang = atan2(y, x);
            if (ang < 0) ang += 2.0 * M_PI;
            if (ring == 0) ang = 0.0;
            pts.push_back({ring, ang, x, y});
        }
    std::stable_sort(pts.begin(), pts.end(), [](const P& a, const P& b) {
        if (a.ring != b.ring) return a.ring < b.ring;
        return a.ang < b.ang;
    });
    out.clear();
    for (const P& p : pts) {
        out.push_back(p.x);
        out.push_back(p.y);
    }
    return static_cast<int>(pts.size());
}

}  // namespace gateau
