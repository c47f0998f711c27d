// Host-side FP64 plan tables (see plan_host.cpp).
#pragma once

#include <string>
#include <vector>

#include "../../include/gateau.h"

namespace gateau {

// Exact SI constants (CODATA 2018).
constexpr double kH = 6.62607015e-34;
constexpr double kKB = 1.380649e-23;
constexpr double kC = 299792458.0;

struct StageSpec {
    int kind;
    double T_K;
    double eta;
    std::vector<double> eta_nu;
    double eps_ref, nu_ref_hz;
    double d_m, n_index, tan_delta, T_refl_K;
    int ar_coated;
};

struct PrimStage {
    std::vector<double> eta;
    bool sky;
    double T;
};

std::vector<double> make_grid(int n, double f_lo, double f_hi);
std::vector<double> make_trapezoid(const std::vector<double>& nu);
double jn_power(double T, double nu);
bool expand_stages(const std::vector<StageSpec>& stages, const std::vector<double>& nu,
                   std::vector<PrimStage>& out, std::string& err);
void collapse_cascade(const std::vector<double>& nu, const std::vector<PrimStage>& prim, double T_atm,
                      double T_cmb, double eta_taper, double rho_surf, double eta_pol, std::vector<double>& c0,
                      std::vector<double>& c1, std::vector<double>& c2);
bool build_filters(int kind, int n_ch, const double* f_c, const double* R, const double* eta_peak,
                   const double* custom, const std::vector<double>& nu, double delta_al_J,
                   std::vector<double>& eta, std::string& err);
int pink_pole_count(double f_min, double f_sample);
void pink_design_channel(double alpha, double A, double f_min, double f_sample, int n_pole, double* a_out,
                         double* r_out, double* d_out);
int hex_offsets(int R_hex, double spacing, std::vector<double>& out);

}  // namespace gateau
