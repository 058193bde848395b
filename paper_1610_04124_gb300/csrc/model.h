// model.h -- host-side construction of the fixed-point stixel model.
#pragma once

#include <stdint.h>

#include <vector>

#include "stixels.h"

namespace stx {

// The "offline" part of the look-up tables (Sec. 3.4): everything that does
// not depend on the input disparities, computed once per parameter set in FP64
// and rounded to the fixed-point grid.
struct HostModel {
    stixels_params_t p;
    int dmax = 0, emax = 0;
    double alpha = 0.0;                 // ground slope in px of disparity per image row
    int32_t c_out = 0, k_sky = 0;
    std::vector<int32_t> k_obj;         // [dmax + 1]
    std::vector<int32_t> g_obj;         // [emax + 1], or [dmax + 1][emax + 1] with variable sigma
    std::vector<int32_t> g_ground, g_sky;          // [emax + 1] (g_ground: constant sigma only)
    bool var_sigma = false;             // sigma_gain != 0: per-disparity / per-row residual tables
    int32_t first[3] = {0, 0, 0};
    int32_t trans[3][3] = {{0}};
    int32_t pen_grav = 0, pen_div = 0, pen_ord = 0;
    int32_t eps_g = 0, eps_d = 0, eps_o = 0;
    int32_t max_finite_prior = 0;       // largest finite prior + penalty sum for one stixel
    int32_t esat[3] = {0, 0, 0};        // saturation residual (Q4) per class: object, ground, sky
    // whole-pixel grid only: object pixel cost of pixel disparity d under model
    // disparity f, cost[f * (dmax + 1) + d] (the paper's LUT_cost); empty otherwise
    std::vector<int32_t> lut_cost;
    // ground estimate only: ground K for every ground code c in [0, 16 dmax]
    // (K depends on the ground disparity only through its clamp to [0, d_range])
    std::vector<int32_t> kg_tab;
};

// Validate params and build the model; returns a stixels_status.
int build_model(const stixels_params_t* p, HostModel* m);

// Per-height row tables: ground-line Q4 disparity and ground K for v = 0..H-1
// (v = 0 is the bottom image row); with variable sigma also the ground
// residual table of every row, g_rows[v * (emax + 1) + e] (else left empty).
// Returns false if a row's table would not reach the outlier branch.
bool build_rows(const HostModel& m, int H, std::vector<int32_t>* fgq, std::vector<int32_t>* k_ground,
                std::vector<int32_t>* g_rows);

// sigma^c at model disparity f for a class whose base sigma is `base`.
double sigma_at(const stixels_params_t& p, double base, double f);

// True if every cost of an H-row column fits the int32 budget (see internal.h).
bool budget_ok(const HostModel& m, int H, const std::vector<int32_t>& k_ground);

void default_params(stixels_params_t* p);

}  // namespace stx
