// model.h -- host-side construction of the fixed-point stixel model.
#pragma once

#include <stdint.h>

#include <vector>

#include "stixels.h"

namespace stx {

// Unrounded model constants (Eq. 3-4 and the priors) for the real-arithmetic
// cost of a solved segmentation.
struct RealModel {
    float c_out = 0.f, k_sky = 0.f, inv_sky = 0.f, inv_ground = 0.f;   // inv = 1 / (2 sigma^2)
    std::vector<float> k_obj, inv_obj;                                  // [dmax + 1]
    double first[3] = {0, 0, 0}, trans[3][3] = {{0}};                   // prior + BIC
    double pen_grav = 0, pen_div = 0, pen_ord = 0;
    double eps_g = 0, eps_d = 0, eps_o16 = 0;
    std::vector<float> rkg_tab;         // ground estimate only: [256 dmax + 1] K at f = c / 256
};

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
    std::vector<int32_t> g_ground, g_sky;          // [emax + 1] (g_ground: the create-time check only)
    bool var_sigma = false;             // sigma_gain != 0: per-disparity residual tables
    int32_t first[3] = {0, 0, 0};
    int32_t trans[3][3] = {{0}};
    int32_t pen_grav = 0, pen_div = 0, pen_ord = 0;
    int32_t ord_off = 0;                // floor(eps_order)
    int32_t max_finite_prior = 0;       // largest finite prior + penalty sum for one stixel
    int32_t pixel_floor = 0;            // no object pixel costs less: min(C_out, every object K)
    int32_t esat[3] = {0, 0, 0};        // saturation residual (Q4) per class: object, ground, sky
    // whole-pixel grid only: object pixel cost of pixel disparity d under model
    // disparity f, cost[f * (dmax + 1) + d] (the paper's LUT_cost); empty otherwise
    std::vector<int32_t> lut_cost;
    // ground estimate only: ground K at every ground disparity c / 256, c in
    // [0, 256 dmax] (an estimated line's disparities are multiples of 1/256
    // px, and K depends on the disparity only through its clamp to [0, d_range])
    std::vector<int32_t> kg_tab;
    // ground estimate only: the 16 ground residual windows of an estimated
    // line (one per 1/256-px phase of 16 f_g), est_gw codes each (RowsDev)
    std::vector<int32_t> est_pool;
    int est_gw = 0;
    // The same model without the fixed-point grid, for the cost report: the
    // per-pixel constants of Eq. 3-4 in FP32, the priors in FP64 (the
    // device gets them in fixed point, RealParams).
    RealModel real;
};

// Validate params and build the model; returns a stixels_status.
int build_model(const stixels_params_t* p, HostModel* m);

// The row tables of the camera's ground line for height H, packed as the
// device reads them (RowsDev): the per-row arrays, then at
// rows_arrays_bytes(H) the rows' residual windows, *gw codes each.  Returns
// false if a row's residual does not reach the outlier cost within dmax px or
// a cost of the line does not fit the fixed-point budget.
bool build_rows(const HostModel& m, int H, std::vector<char>* block, int* gw);

// sigma^c at model disparity f for a class whose base sigma is `base`.
double sigma_at(const stixels_params_t& p, double base, double f);

// True if every cost of an H-row column fits the int32 budget (see internal.h);
// k_ground: the ground K of its rows.
bool budget_ok(const HostModel& m, int H, const int32_t* k_ground);

void default_params(stixels_params_t* p);

}  // namespace stx
