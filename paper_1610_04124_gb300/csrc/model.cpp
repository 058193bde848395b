// model.cpp -- the input-independent ("offline") part of the stixel model
// (Sec. 3.4), built once per parameter set on the host in FP64 and rounded to
// the fixed-point grid used by the kernels.
//
// Sensor model (Eq. 3) and per-pixel cost (Eq. 4):
//   cost(d | f) = min( C_out , K(f) + (d - f)^2 / (2 sigma^2) )
//   C_out = ln d_range - ln p_out
//   K(f)  = ln A_norm(f) + ln(sigma sqrt(2 pi)) - ln(1 - p_out)
//   A_norm(f) = Phi((d_range - f)/sigma) - Phi(-f/sigma), f clamped to [0, d_range]
// with d_range = dmax and sigma a per-class constant (the paper's noise model
// sigma^c(f, v) is not specified further).  The class models (Sec. 3.1): object
// f = rounded mean disparity of the stixel; ground f(v) = alpha (v_hor - v), i.e.
// alpha (r - horizon_row) at image row r, alpha = baseline cos(pitch) / height,
// put on the 1/16-px grid; sky f = 0.
//
// Fixed point: each of C_out, K and the residual term is rounded to the
// nearest multiple of 2^-12 (halves away from zero) and stored in 2^-14 units
// (so as a multiple of 4).  The residual term is tabulated over the Q4
// residual e = |q - 16 f| in [0, 16 dmax]; larger residuals clamp to the last
// entry, which create() checks is already past the outlier branch.  The
// expressions below are evaluated in IEEE FP64 exactly as written (the build
// disables floating-point contraction), which makes the tables reproducible.
#include "model.h"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace stx {

namespace {

double std_normal_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

double norm_mass(double f, double sigma, double d_range)
{
    double fc = f < 0.0 ? 0.0 : (f > d_range ? d_range : f);
    return std_normal_cdf((d_range - fc) / sigma) - std_normal_cdf((0.0 - fc) / sigma);
}

double gauss_const(double f, double sigma, double p_out, double d_range)
{
    return log(norm_mass(f, sigma, d_range)) + log(sigma * sqrt(2.0 * M_PI)) - log(1.0 - p_out);
}

double resid(double dpx, double sigma) { return dpx * dpx / (2.0 * sigma * sigma); }

// Residual terms are capped at 65536 cost units before rounding: every capped
// entry is far past the outlier branch (C_out - K is at most a few hundred),
// so min(C_out, K + term) is unchanged and the table stays inside int32.
double resid_capped(double dpx, double sigma)
{
    double r = resid(dpx, sigma);
    return r < 65536.0 ? r : 65536.0;
}

// multiple of 2^-12, in 2^-14 units
int32_t to_fixed(double x) { return (int32_t)(4 * llround(4096.0 * x)); }

bool finite_pos(float x) { return std::isfinite(x) && x > 0.0f; }

bool sigma_ok(float x) { return finite_pos(x) && x <= 1000.0f; }

// a prior: >= 0, and finite <= 1000 or +inf
bool prior_ok(float x) { return !std::isnan(x) && x >= 0.0f && (std::isinf(x) || x <= 1000.0f); }

int32_t fixed_prior(double x) { return std::isinf(x) ? kBig : to_fixed(x); }

// The reach ER (Q4 codes) of a ground residual window: the smallest e with
// kmin + G(e / 16) >= C_out (G the residual term on the grid), so that a pixel
// e / 16 px or more from the line costs C_out whatever its K (>= kmin); -1 if
// that takes more than emax codes (dmax px).
int ground_reach(double sigma, int32_t kmin, int32_t c_out, int emax)
{
    for (int e = 0; e <= emax; ++e)
        if ((int64_t)kmin + to_fixed(resid_capped(e / 16.0, sigma)) >= c_out) return e;
    return -1;
}

}  // namespace

void default_params(stixels_params_t* p)
{
    std::memset(p, 0, sizeof(*p));
    p->focal_px = 700.0f;
    p->baseline_m = 0.3f;
    p->camera_height_m = 1.2f;
    p->pitch_rad = 0.0f;
    p->horizon_row = 40;
    p->stixel_width = 5;
    p->dmax = 64;
    p->p_out = 0.05f;
    p->sigma_ground = p->sigma_object = p->sigma_sky = 1.0f;
    // first stixel: object, ground, sky
    p->prior_first[0] = 1.0f; p->prior_first[1] = 0.2f; p->prior_first[2] = 5.0f;
    // [above][below]; ground above ground / sky and sky above sky are impossible
    const float inf = INFINITY;
    const float t[3][3] = {{1.5f, 1.0f, 4.0f}, {1.5f, inf, inf}, {0.5f, 0.5f, inf}};
    std::memcpy(p->prior_trans, t, sizeof(t));
    p->cost_new_stixel = 3.0f;
    p->cost_gravity = 2.0f; p->eps_gravity = 1.0f;
    p->cost_diving = 10.0f; p->eps_diving = 1.0f;
    p->cost_order = 2.0f; p->eps_order = 0.0f;
    p->reduce_mode = 0;
    p->max_stixels_per_col = 64;
    p->pixel_grid = 0;
    p->sigma_gain = 0.0f;
    p->sigma_mid = 32.0f;
    p->sigma_width = 8.0f;
    p->ground_estimate = 0;
    p->global_map = 0;
}

double sigma_at(const stixels_params_t& p, double base, double f)
{
    if (p.sigma_gain == 0.0f) return base;
    const double s = 1.0 / (1.0 + exp(-(f - (double)p.sigma_mid) / (double)p.sigma_width));
    return base * (1.0 + (double)p.sigma_gain * s);
}

int build_model(const stixels_params_t* p, HostModel* m)
{
    if (!p || !m) return STIXELS_E_INVALID_ARG;
    if (p->dmax < 1 || p->dmax > STIXELS_MAX_DMAX) return STIXELS_E_INVALID_ARG;
    if (p->stixel_width < 1 || p->stixel_width > STIXELS_MAX_STIXEL_WIDTH) return STIXELS_E_INVALID_ARG;
    if (!(p->p_out > 0.0f && p->p_out < 1.0f)) return STIXELS_E_INVALID_ARG;
    if (!sigma_ok(p->sigma_ground) || !sigma_ok(p->sigma_object) || !sigma_ok(p->sigma_sky))
        return STIXELS_E_INVALID_ARG;
    if (!finite_pos(p->camera_height_m) || !std::isfinite(p->baseline_m) || !std::isfinite(p->pitch_rad) ||
        std::fabs(p->pitch_rad) >= 1.5f)
        return STIXELS_E_INVALID_ARG;
    for (int c = 0; c < 3; ++c) {
        if (!prior_ok(p->prior_first[c])) return STIXELS_E_INVALID_ARG;
        for (int q = 0; q < 3; ++q)
            if (!prior_ok(p->prior_trans[c][q])) return STIXELS_E_INVALID_ARG;
    }
    if (!prior_ok(p->cost_new_stixel) || std::isinf(p->cost_new_stixel)) return STIXELS_E_INVALID_ARG;
    // the data-dependent penalties must be finite: a feasible segmentation then
    // never needs more than three stixels to reach any class, which bounds every
    // feasible cost (see budget_ok)
    for (float c : {p->cost_gravity, p->cost_diving, p->cost_order})
        if (!prior_ok(c) || std::isinf(c)) return STIXELS_E_INVALID_ARG;
    const float eps[3] = {p->eps_gravity, p->eps_diving, p->eps_order};
    for (float e : eps)
        if (!std::isfinite(e) || std::fabs(e) > 100.0f) return STIXELS_E_INVALID_ARG;
    // gravity (f above the ground line + eps) and diving (f below it - eps) must
    // exclude each other
    if (p->eps_gravity < 0.0f || p->eps_diving < 0.0f) return STIXELS_E_INVALID_ARG;
    if (p->reduce_mode != 0 && p->reduce_mode != 1) return STIXELS_E_INVALID_ARG;
    if (p->pixel_grid != 0 && p->pixel_grid != 1) return STIXELS_E_INVALID_ARG;
    if (!(p->sigma_gain > -1.0f && p->sigma_gain <= 10.0f)) return STIXELS_E_INVALID_ARG;
    if (p->sigma_gain != 0.0f && !(p->sigma_width > 0.0f && std::isfinite(p->sigma_width) &&
                                   std::isfinite(p->sigma_mid)))
        return STIXELS_E_INVALID_ARG;
    if (p->ground_estimate != 0 && p->ground_estimate != 1) return STIXELS_E_INVALID_ARG;
    if (p->ground_estimate && p->sigma_gain != 0.0f) return STIXELS_E_INVALID_ARG;
    if (p->global_map != 0 && p->global_map != 1) return STIXELS_E_INVALID_ARG;
    if (p->max_stixels_per_col < 1 || p->max_stixels_per_col > STIXELS_MAX_HEIGHT) return STIXELS_E_INVALID_ARG;

    m->p = *p;
    m->dmax = p->dmax;
    m->emax = 16 * p->dmax;
    const double d_range = (double)p->dmax;
    const double p_out = (double)p->p_out;
    const double s_obj = (double)p->sigma_object, s_gnd = (double)p->sigma_ground, s_sky = (double)p->sigma_sky;

    m->c_out = to_fixed(log(d_range) - log(p_out));
    m->var_sigma = p->sigma_gain != 0.0f;
    const int F = m->dmax + 1, E = m->emax + 1;
    // sigma^c(f) (Eq. 3): per object disparity, and the sky's at f = 0; the
    // ground's depends on the row (build_rows)
    std::vector<double> so(F);
    m->k_obj.resize(F);
    for (int f = 0; f < F; ++f) {
        so[f] = sigma_at(*p, s_obj, (double)f);
        m->k_obj[f] = to_fixed(gauss_const((double)f, so[f], p_out, d_range));
    }
    const double s_sky_f = sigma_at(*p, s_sky, 0.0);
    m->k_sky = to_fixed(gauss_const(0.0, s_sky_f, p_out, d_range));
    m->g_obj.resize(m->var_sigma ? (size_t)F * E : (size_t)E);
    m->g_ground.resize(E);
    m->g_sky.resize(E);
    for (int e = 0; e < E; ++e) {
        const double dpx = e / 16.0;
        if (!m->var_sigma) m->g_obj[e] = to_fixed(resid_capped(dpx, s_obj));
        m->g_ground[e] = to_fixed(resid_capped(dpx, s_gnd));
        m->g_sky[e] = to_fixed(resid_capped(dpx, s_sky_f));
    }
    if (m->var_sigma)
        for (int f = 0; f < F; ++f)
            for (int e = 0; e < E; ++e) m->g_obj[(size_t)f * E + e] = to_fixed(resid_capped(e / 16.0, so[f]));
    if (!m->var_sigma) {
        // the residual table must reach the outlier branch before it ends, for
        // every class and every K (K is smallest at the clamped ends of [0, d_range])
        const int32_t kmin[3] = {to_fixed(gauss_const(0.0, s_obj, p_out, d_range)),
                                 to_fixed(gauss_const(0.0, s_gnd, p_out, d_range)),
                                 to_fixed(gauss_const(0.0, s_sky, p_out, d_range))};
        const int32_t glast[3] = {m->g_obj[m->emax], m->g_ground[m->emax], m->g_sky[m->emax]};
        for (int c = 0; c < 3; ++c)
            if ((int64_t)kmin[c] + glast[c] < m->c_out) return STIXELS_E_INVALID_ARG;
        // first residual from which every pixel of the class costs C_out (the
        // tables are non-decreasing in e, and K >= kmin)
        const std::vector<int32_t>* gtab[3] = {&m->g_obj, &m->g_ground, &m->g_sky};
        for (int c = 0; c < 3; ++c) {
            int e = 0;
            while (e < m->emax && (int64_t)kmin[c] + (*gtab[c])[e] < m->c_out) ++e;
            m->esat[c] = e;
        }
    } else {
        // per disparity: the row of every f must reach the outlier branch; esat
        // of the objects is the largest first saturated residual over f
        int es = 0;
        for (int f = 0; f < F; ++f) {
            const int32_t* g = m->g_obj.data() + (size_t)f * E;
            if ((int64_t)m->k_obj[f] + g[m->emax] < m->c_out) return STIXELS_E_INVALID_ARG;
            int e = 0;
            while (e < m->emax && (int64_t)m->k_obj[f] + g[e] < m->c_out) ++e;
            es = std::max(es, e);
        }
        m->esat[0] = es;
        m->esat[1] = m->emax;                          // ground rows are checked per height
        if ((int64_t)m->k_sky + m->g_sky[m->emax] < m->c_out) return STIXELS_E_INVALID_ARG;
        int e = 0;
        while (e < m->emax && (int64_t)m->k_sky + m->g_sky[e] < m->c_out) ++e;
        m->esat[2] = e;
    }

    m->alpha = (double)p->baseline_m * cos((double)p->pitch_rad) / (double)p->camera_height_m;

    const double bic = (double)p->cost_new_stixel;
    int32_t maxp = 0;
    for (int c = 0; c < 3; ++c) {
        m->first[c] = fixed_prior((double)p->prior_first[c] + bic);
        if (m->first[c] < kBig && m->first[c] > maxp) maxp = m->first[c];
        for (int q = 0; q < 3; ++q) {
            m->trans[c][q] = fixed_prior((double)p->prior_trans[c][q] + bic);
            if (m->trans[c][q] < kBig && m->trans[c][q] > maxp) maxp = m->trans[c][q];
        }
    }
    m->pen_grav = fixed_prior((double)p->cost_gravity);
    m->pen_div = fixed_prior((double)p->cost_diving);
    m->pen_ord = fixed_prior((double)p->cost_order);
    m->max_finite_prior = maxp + m->pen_grav + m->pen_div + m->pen_ord;
    // an object pixel costs min(C_out, K(f) + G) >= min(C_out, K(f)) (and the
    // whole-pixel grid's LUT_cost entries are those same values): the floor
    // the DP's tile bound uses is the least of C_out and every object K
    {
        int32_t fl = m->c_out;
        for (int32_t k : m->k_obj) fl = std::min(fl, k);
        m->pixel_floor = fl;
    }
    // 16 f > 16 f' + 16 eps  <=>  f - f' > floor(eps) for integer f, f'
    m->ord_off = (int32_t)floor((double)p->eps_order);
    // the same constants without the grid (the cost report of a solved column)
    RealModel& r = m->real;
    r.c_out = (float)(log(d_range) - log(p_out));
    r.k_obj.resize(F);
    r.inv_obj.resize(F);
    for (int f = 0; f < F; ++f) {
        r.k_obj[f] = (float)gauss_const((double)f, so[f], p_out, d_range);
        r.inv_obj[f] = (float)(1.0 / (2.0 * so[f] * so[f]));
    }
    r.k_sky = (float)gauss_const(0.0, s_sky_f, p_out, d_range);
    r.inv_sky = (float)(1.0 / (2.0 * s_sky_f * s_sky_f));
    r.inv_ground = (float)(1.0 / (2.0 * s_gnd * s_gnd));
    for (int c = 0; c < 3; ++c) {
        r.first[c] = (double)p->prior_first[c] + bic;
        for (int q = 0; q < 3; ++q) r.trans[c][q] = (double)p->prior_trans[c][q] + bic;
    }
    r.pen_grav = (double)p->cost_gravity;
    r.pen_div = (double)p->cost_diving;
    r.pen_ord = (double)p->cost_order;
    r.eps_g = (double)p->eps_gravity;
    r.eps_d = (double)p->eps_diving;
    r.eps_o16 = 16.0 * (double)p->eps_order;
    m->kg_tab.clear();
    r.rkg_tab.clear();
    m->est_pool.clear();
    m->est_gw = 0;
    if (p->ground_estimate) {
        const int nc = 256 * m->dmax + 1;
        m->kg_tab.resize(nc);
        r.rkg_tab.resize(nc);
        int32_t kmin = INT32_MAX;
        for (int c = 0; c < nc; ++c) {
            const double k = gauss_const(c / 256.0, s_gnd, p_out, d_range);
            m->kg_tab[c] = to_fixed(k);
            r.rkg_tab[c] = (float)k;
            kmin = std::min(kmin, m->kg_tab[c]);
        }
        // the windows of an estimated line f_g = x / 256: at code q = (x >> 4)
        // - ER + j the residual is ((16 (j - ER) - (x & 15)) / 256)^2 / (2
        // sigma^2), so it depends only on j and the phase x & 15
        const int er = ground_reach(s_gnd, kmin, m->c_out, m->emax);
        if (er < 0) return STIXELS_E_INVALID_ARG;
        m->est_gw = 2 * er + 2;
        m->est_pool.resize((size_t)16 * m->est_gw);
        for (int ph = 0; ph < 16; ++ph)
            for (int j = 0; j < m->est_gw; ++j)
                m->est_pool[(size_t)ph * m->est_gw + j] =
                    to_fixed(resid_capped((double)(16 * (j - er) - ph) / 256.0, s_gnd));
    }
    // whole-pixel grid: the object pixel cost of every (model disparity f,
    // pixel disparity d) pair, the same value as the per-pixel formula at the
    // Q4 residual 16 |d - f| (paper Sec. 3.4's LUT_cost, computed off-line)
    m->lut_cost.clear();
    if (p->pixel_grid) {
        m->lut_cost.resize((size_t)F * F);
        for (int f = 0; f < F; ++f)
            for (int d = 0; d < F; ++d) {
                const int e = std::min(16 * std::abs(d - f), m->var_sigma ? m->emax : m->esat[0]);
                const int32_t g = m->var_sigma ? m->g_obj[(size_t)f * (m->emax + 1) + e] : m->g_obj[e];
                m->lut_cost[(size_t)f * F + d] = std::min(m->c_out, m->k_obj[f] + g);
            }
    }
    return STIXELS_OK;
}

bool build_rows(const HostModel& m, int H, std::vector<char>* block, int* gw)
{
    const double d_range = (double)m.dmax;
    const double p_out = (double)m.p.p_out;
    const double s_gnd = (double)m.p.sigma_ground;
    std::vector<double> fgv(H), sgv(H);
    std::vector<int32_t> kgv(H);
    int er = 0;
    for (int v = 0; v < H; ++v) {
        const int r = H - 1 - v;                       // image row of bottom-up row v
        fgv[v] = m.alpha * (double)(r - m.p.horizon_row);
        sgv[v] = sigma_at(m.p, s_gnd, fgv[v]);
        kgv[v] = to_fixed(gauss_const(fgv[v], sgv[v], p_out, d_range));
        const int e = ground_reach(sgv[v], kgv[v], m.c_out, m.emax);
        if (e < 0) return false;
        er = std::max(er, e);
    }
    if (!budget_ok(m, H, kgv.data())) return false;
    // a handle that estimates its ground swaps these rows for a frame's when
    // something votes: both use one window size (the estimate's reach, taken
    // over every K, is the larger)
    if (m.p.ground_estimate) er = std::max(er, (m.est_gw - 2) / 2);
    *gw = 2 * er + 2;
    const size_t arrays = rows_arrays_bytes(H);
    block->assign(arrays + sizeof(int32_t) * (size_t)H * *gw, 0);
    double* fg = reinterpret_cast<double*>(block->data());
    int32_t* kg = reinterpret_cast<int32_t*>(fg + H);
    int32_t* thr = kg + H;
    int32_t* gf = kg + 2 * H;
    int32_t* goff = kg + 3 * H;
    float* rkg = reinterpret_cast<float*>(kg + 4 * H);
    float* rinv = rkg + H;
    float* rdg = rkg + 2 * H;
    int32_t* pool = reinterpret_cast<int32_t*>(block->data() + arrays);
    for (int v = 0; v < H; ++v) {
        const double f = fgv[v];
        const int32_t g = (int32_t)floor(16.0 * f);
        fg[v] = f;
        kg[v] = kgv[v];
        thr[v] = pack_thresholds(f, (double)m.p.eps_gravity, (double)m.p.eps_diving);
        gf[v] = g;
        goff[v] = v * *gw;
        rkg[v] = (float)gauss_const(f, sgv[v], p_out, d_range);
        rinv[v] = (float)(1.0 / (2.0 * sgv[v] * sgv[v]));
        rdg[v] = (float)(f - (double)g / 16.0);
        // the window: codes q = g - ER .. g + ER + 1, residual of (q / 16 - f_g)
        for (int j = 0; j < *gw; ++j) {
            const int q = g - er + j;
            pool[(size_t)v * *gw + j] = to_fixed(resid_capped((double)q / 16.0 - f, sgv[v]));
        }
    }
    return true;
}

// A feasible cell of the cost table is reached by some segmentation of at most
// three stixels (one per class change), so every feasible cost is below
// H * max|pixel cost| + 3 * (largest prior of one stixel).  Keeping that below
// 2^28 units keeps feasible costs below the 2^29 "infeasible" marker and every
// candidate sum (cost <= 2^29, transition <= 2^29, penalty, data) inside int32.
bool budget_ok(const HostModel& m, int H, const int32_t* k_ground)
{
    int64_t kmin = m.k_sky;
    for (int32_t k : m.k_obj) kmin = k < kmin ? k : kmin;
    for (int v = 0; v < H; ++v) kmin = k_ground[v] < kmin ? k_ground[v] : kmin;
    int64_t per_pixel = m.c_out > -kmin ? m.c_out : -kmin;
    int64_t worst = (int64_t)H * per_pixel + 3 * (int64_t)m.max_finite_prior;
    return worst < kFiniteBudget;
}

}  // namespace stx
