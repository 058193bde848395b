/*
 * oracle.c -- plain, slow, obviously-correct CPU reference of multi-stixel
 * estimation as described in "GPU-accelerated real-time stixel computation"
 * (Hernandez-Juarez et al., arXiv 1610.04124).
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg are the only users of this file.  The CUDA
 * library never links, loads or includes it, and this file includes nothing
 * of the library: the two share no code, header, table or constant generator.
 *
 * Per stixel-width column it computes, in the paper's order:
 *   1. the column reduction of Sec. 5.1 (median of the s pixels of a row by
 *      default, or their mean as the paper states), after clamping each pixel
 *      to [0, dmax] and putting it on the 1/16-pixel grid ("Q4"); with
 *      pixel_grid set, the reduced value is then rounded to whole pixels, the
 *      integer disparities of Sec. 3.4's LUT_cost variant;
 *   2. the per-pixel data cost of Eq. 4 for the object, ground and sky models
 *      of Sec. 3.1, with the sensor model of Eq. 3;
 *   3. prefix sums of those costs and of the disparities (Sec. 3.4);
 *   4. the dynamic program of Eq. 5 (base case) and Eq. 6 (recurrence) for the
 *      three classes, evaluated plainly: for every end row k, every class c,
 *      every start row b <= k and every previous class p;
 *   5. backtracking from the top row through the index table (Sec. 3.3).
 * It also enumerates every segmentation of short columns (brute force) and
 * re-evaluates the cost of a given segmentation from direct per-pixel sums.
 *
 * Two arithmetic modes:
 *   quantize = 1  every per-pixel cost term (C_out, the normalisation
 *                 constant K, the squared-residual term) and every prior is
 *                 put on the 2^-12 cost grid before use.  All sums are then
 *                 exact in FP64, so ties are exact and the tie-break below
 *                 decides them.  This is the arithmetic the CUDA library's DP
 *                 decides in (int32).  The ground line and the gravity,
 *                 diving and ordering thresholds are the model's own, not
 *                 rounded, in both modes.
 *   quantize = 0  the same formulation with plain FP64 reals: the paper's
 *                 arithmetic, which the library's reported costs follow.
 *
 * Readings of the paper where it is silent or ambiguous (all restated in the
 * project's design notes):
 *   - row index v = 0 is the bottom pixel of the column (Eq. 5 describes the
 *     base case as the single pixel at the bottom; backtracking starts at the
 *     top row); stixel bounds are 0 <= v_b <= v_t <= h-1;
 *   - prefix arrays carry a leading zero, so LUT[v_b - 1] at v_b = 0 is 0;
 *   - ground model f(v) = alpha (v_horizon - v) (Sec. 3.1) with
 *     alpha = baseline cos(pitch) / camera height, i.e. in image rows r
 *     (0 = top) f = alpha (r - horizon_row);
 *   - sigma^c is a per-class constant, or with sigma_gain set a logistic in
 *     the model disparity (the paper names a sigmoid but not its form; see
 *     or_params_t); A_norm is the mass of the Gaussian
 *     N(f, sigma^2) on [0, d_range] with f clamped to [0, d_range];
 *     d_range = dmax;
 *   - Eq. 4's min(., .) is used as printed;
 *   - the object disparity f is the mean Q4 disparity of the stixel rounded
 *     half up to an integer: f = floor((S + 8 n) / (16 n));
 *   - priors (Sec. 3 constraints 1-5; the paper defers their values to
 *     Pfeiffer's thesis): BIC cost per stixel, first-stixel cost per class,
 *     class-transition costs (INFINITY = forbidden), gravity and diving
 *     penalties for an object directly above ground (compared with the ground
 *     disparity at the object's base row), ordering penalty for an object
 *     directly above an object whose disparity is lower by more than eps;
 *   - the DP keeps, per end row and class, only the best stixel (Eq. 6 links
 *     candidates to ob^{k-1}, gr^{k-1}, sk^{k-1}); with the ordering penalty
 *     on this is the paper's DP, not the global MAP (global_map = 1 computes
 *     the global MAP instead);
 *   - ties within a cell are broken by (cost, previous class, start row) in
 *     lexicographic order, classes ordered object < ground < sky < none (the
 *     first stixel); the final class at the top row is chosen in the order
 *     object < ground < sky.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OBJECT 0
#define OR_GROUND 1
#define OR_SKY 2
#define OR_NONE 3

#define OR_OK 0
#define OR_E_ARG 1
#define OR_E_MEM 2
#define OR_E_INFEASIBLE 3
#define OR_E_CAPACITY 4

/* Camera, sensor-model and prior parameters (single precision, as a caller
 * would hand them to the library; every derived quantity is FP64). */
typedef struct {
    float focal_px, baseline_m, camera_height_m, pitch_rad;
    int32_t horizon_row, stixel_width, dmax;
    float p_out, sigma_ground, sigma_object, sigma_sky;
    float prior_first[3];       /* -ln P(class of the bottom stixel): object, ground, sky */
    float prior_trans[3][3];    /* [above][below] -ln P; INFINITY = forbidden */
    float cost_new_stixel;      /* BIC cost, added once per stixel */
    float cost_gravity, eps_gravity, cost_diving, eps_diving, cost_order, eps_order;
    int32_t reduce_mode;        /* 0 = median, 1 = mean */
    int32_t quantize;           /* 1 = fixed grids (the library's arithmetic), 0 = plain reals */
    int32_t pixel_grid;         /* 1 = reduced disparities rounded to whole pixels (Sec. 3.4's
                                   integer LUT_cost variant), 0 = kept on the 1/16-px grid */
    /* disparity-dependent noise (Eq. 3's sigma^c(f, v), "a sigmoid function"):
     * sigma^c(f) = sigma_c (1 + sigma_gain / (1 + exp(-(f - sigma_mid) / sigma_width))),
     * f the model disparity (object: f; ground: the ground line at row v; sky: 0);
     * sigma_gain = 0 is the constant-sigma model */
    float sigma_gain, sigma_mid, sigma_width;
    /* 1 = the ground line comes from the frame itself (or_ground_estimate on
     * its reduced codes) instead of the camera parameters */
    int32_t ground_estimate;
    /* 1 = the global MAP over all segmentations with the ordering prior exact:
     * the object state carries the disparity of its stixel (Eq. 6 keeps only
     * the best stixel per row and class, which makes the ordering prior an
     * approximation); 0 = the paper's DP */
    int32_t global_map;
} or_params_t;

typedef struct {
    int32_t v_bottom, v_top;   /* bottom-up rows, inclusive */
    int32_t cls;               /* OR_OBJECT / OR_GROUND / OR_SKY */
    int32_t f;                 /* rounded mean disparity (integer px) */
    int64_t sum_q;             /* sum of the Q4 disparities over the stixel */
    double disparity;          /* exact mean: sum_q / (16 n) */
} or_stixel_t;

/* Derived model for one column height H. */
typedef struct {
    int H, dmax, quantize;
    double c_out;              /* ln d_range - ln p_out */
    double *k_obj;             /* [dmax+1]: K for the object model at integer f */
    double *fg;                /* [H]: ground-model disparity at bottom-up row v */
    double *k_ground;          /* [H] */
    double k_sky;
    double sigma[3];           /* base sigma per class */
    double *sig_obj;           /* [dmax+1]: object sigma at integer f */
    double *sig_gnd;           /* [H]: ground sigma at row v */
    double sig_sky;
    double first[3];           /* first-stixel prior + BIC (INFINITY = forbidden) */
    double trans[3][3];        /* transition prior + BIC, [above][below] */
    double pen_grav, pen_div, pen_ord;
    double *g_hi, *g_lo;       /* [H]: gravity / diving thresholds on 16 f, at the object's base */
    double ord_eps16;          /* ordering threshold offset on 16 f */
} or_model_t;

/* ---------------------------------------------------------------- grids */

/* nearest point of the 2^-12 cost grid (halves away from zero) */
static double cost_grid(double x) { return (double)llround(4096.0 * x) / 4096.0; }

static double maybe_grid(const or_model_t* m, double x)
{
    if (!m->quantize || isinf(x)) return x;
    return cost_grid(x);
}

/* Q4 code of one input pixel: clamp to [0, dmax] (NaN -> 0), then round
 * 16 d to the nearest integer, halves to even. */
static int32_t q4_of(float d, int dmax)
{
    if (!(d > 0.0f)) return 0;                  /* also catches NaN */
    if (d >= (float)dmax) return 16 * dmax;
    return (int32_t)nearbyintf(16.0f * d);
}

/* ------------------------------------------------------- sensor model (Eq. 3, Eq. 4) */

/* standard normal CDF */
static double Phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* A_norm: probability mass of N(f, sigma^2) on [0, d_range], f clamped to [0, d_range] */
static double a_norm(double f, double sigma, double d_range)
{
    double fc = f < 0.0 ? 0.0 : (f > d_range ? d_range : f);
    return Phi((d_range - fc) / sigma) - Phi((0.0 - fc) / sigma);
}

/* the constant part of the Gaussian branch of Eq. 4:
 * log(A_norm) + log(sigma sqrt(2 pi)) - log(1 - p_out) */
static double k_const(double f, double sigma, double p_out, double d_range)
{
    return log(a_norm(f, sigma, d_range)) + log(sigma * sqrt(2.0 * M_PI)) - log(1.0 - p_out);
}

/* the residual part of Eq. 4: (d - f)^2 / (2 sigma^2) */
static double resid_term(double dpx, double sigma) { return dpx * dpx / (2.0 * sigma * sigma); }

/* Eq. 4 for one pixel: min(uniform branch, Gaussian branch), each term on the grid when quantizing. */
static double pixel_cost(const or_model_t* m, int cls, int v, int32_t q, int f)
{
    double d = q / 16.0, K, r;
    if (cls == OR_OBJECT) {
        K = m->k_obj[f];
        r = resid_term(d - (double)f, m->sig_obj[f]);
    } else if (cls == OR_GROUND) {
        K = m->k_ground[v];
        r = resid_term(d - m->fg[v], m->sig_gnd[v]);
    } else {
        K = m->k_sky;
        r = resid_term(d, m->sig_sky);
    }
    double g = maybe_grid(m, K) + maybe_grid(m, r);
    double c = maybe_grid(m, m->c_out);
    return g < c ? g : c;
}

/* rounded mean of a stixel: floor((S + 8 n) / (16 n)), S = sum of Q4 codes, n rows */
static int mean_f(int64_t S, int n) { return (int)((S + 8 * (int64_t)n) / (16 * (int64_t)n)); }

/* ------------------------------------------------------------------- model */

static void model_free(or_model_t* m)
{
    free(m->k_obj); free(m->fg); free(m->k_ground); free(m->g_hi); free(m->g_lo);
    free(m->sig_obj); free(m->sig_gnd);
    memset(m, 0, sizeof(*m));
}

static int check_params(const or_params_t* p)
{
    if (p->dmax < 1 || p->dmax > 2047) return OR_E_ARG;
    if (!(p->p_out > 0.0f && p->p_out < 1.0f)) return OR_E_ARG;
    if (!(p->sigma_ground > 0.0f && p->sigma_object > 0.0f && p->sigma_sky > 0.0f)) return OR_E_ARG;
    if (!(p->camera_height_m > 0.0f)) return OR_E_ARG;
    if (p->stixel_width < 1) return OR_E_ARG;
    if (!(p->sigma_gain > -1.0f && p->sigma_gain <= 10.0f)) return OR_E_ARG;
    if (p->sigma_gain != 0.0f && !(p->sigma_width > 0.0f && isfinite(p->sigma_mid))) return OR_E_ARG;
    return OR_OK;
}

/* sigma^c at model disparity f (base = the class's sigma) */
static double sigma_at(const or_params_t* p, double base, double f)
{
    if (p->sigma_gain == 0.0f) return base;
    double s = 1.0 / (1.0 + exp(-(f - (double)p->sigma_mid) / (double)p->sigma_width));
    return base * (1.0 + (double)p->sigma_gain * s);
}

/* The model for height H; line_k > 0 replaces the camera's ground line by
 * f(r) = (line_k / 256) (r - line_h) (an estimate from the frame). */
static int model_build_line(const or_params_t* p, int H, int line_k, int line_h, or_model_t* m);

static int model_build(const or_params_t* p, int H, or_model_t* m) { return model_build_line(p, H, 0, 0, m); }

static int model_build_line(const or_params_t* p, int H, int line_k, int line_h, or_model_t* m)
{
    memset(m, 0, sizeof(*m));
    int rc = check_params(p);
    if (rc) return rc;
    if (H < 1) return OR_E_ARG;
    m->H = H;
    m->dmax = p->dmax;
    m->quantize = p->quantize ? 1 : 0;
    const double d_range = (double)p->dmax;
    const double p_out = (double)p->p_out;
    m->sigma[OR_OBJECT] = (double)p->sigma_object;
    m->sigma[OR_GROUND] = (double)p->sigma_ground;
    m->sigma[OR_SKY] = (double)p->sigma_sky;
    m->c_out = log(d_range) - log(p_out);

    m->k_obj = (double*)malloc(sizeof(double) * (size_t)(p->dmax + 1));
    m->fg = (double*)malloc(sizeof(double) * (size_t)H);
    m->k_ground = (double*)malloc(sizeof(double) * (size_t)H);
    m->g_hi = (double*)malloc(sizeof(double) * (size_t)H);
    m->g_lo = (double*)malloc(sizeof(double) * (size_t)H);
    m->sig_obj = (double*)malloc(sizeof(double) * (size_t)(p->dmax + 1));
    m->sig_gnd = (double*)malloc(sizeof(double) * (size_t)H);
    if (!m->k_obj || !m->fg || !m->k_ground || !m->g_hi || !m->g_lo || !m->sig_obj || !m->sig_gnd) {
        model_free(m);
        return OR_E_MEM;
    }

    for (int f = 0; f <= p->dmax; ++f) {
        m->sig_obj[f] = sigma_at(p, m->sigma[OR_OBJECT], (double)f);
        m->k_obj[f] = k_const((double)f, m->sig_obj[f], p_out, d_range);
    }
    m->sig_sky = sigma_at(p, m->sigma[OR_SKY], 0.0);
    m->k_sky = k_const(0.0, m->sig_sky, p_out, d_range);

    /* ground line: image row r = H-1-v; f = alpha (r - horizon) */
    const double alpha = (double)p->baseline_m * cos((double)p->pitch_rad) / (double)p->camera_height_m;
    for (int v = 0; v < H; ++v) {
        int r = H - 1 - v;
        /* the ground model's own disparity at the row, in both modes: the grids
         * apply to cost terms, not to the model or to the thresholds below */
        double fg = line_k > 0 ? (double)line_k * (double)(r - line_h) / 256.0 : alpha * (double)(r - p->horizon_row);
        m->g_hi[v] = 16.0 * (fg + (double)p->eps_gravity);
        m->g_lo[v] = 16.0 * (fg - (double)p->eps_diving);
        m->fg[v] = fg;
        m->sig_gnd[v] = sigma_at(p, m->sigma[OR_GROUND], fg);
        m->k_ground[v] = k_const(fg, m->sig_gnd[v], p_out, d_range);
    }
    m->ord_eps16 = 16.0 * (double)p->eps_order;

    const double bic = (double)p->cost_new_stixel;
    for (int c = 0; c < 3; ++c) {
        m->first[c] = maybe_grid(m, (double)p->prior_first[c] + bic);
        for (int q = 0; q < 3; ++q) m->trans[c][q] = maybe_grid(m, (double)p->prior_trans[c][q] + bic);
    }
    m->pen_grav = maybe_grid(m, (double)p->cost_gravity);
    m->pen_div = maybe_grid(m, (double)p->cost_diving);
    m->pen_ord = maybe_grid(m, (double)p->cost_order);
    return OR_OK;
}

/* prior of stixel (c, starting at b, rounded mean f) directly above a stixel of
 * class p whose rounded mean is f_below (only used for object above object) */
static double pair_prior(const or_model_t* m, int c, int p, int b, int f, int f_below)
{
    double pr = m->trans[c][p];
    if (c == OR_OBJECT && p == OR_GROUND) {
        if (16.0 * f > m->g_hi[b]) pr += m->pen_grav;     /* gravity: object nearer than the ground at its base */
        if (16.0 * f < m->g_lo[b]) pr += m->pen_div;      /* diving: object behind the ground at its base */
    }
    if (c == OR_OBJECT && p == OR_OBJECT) {
        if (16.0 * f > 16.0 * f_below + m->ord_eps16) pr += m->pen_ord;   /* ordering */
    }
    return pr;
}

/* ------------------------------------------------------------- 1. reduction */

/* Column reduction + transpose (Sec. 5.1).  disp: H x W row-major, row 0 = top.
 * q: ncols x H, column c at q[c*H + v] with v = H-1-r (bottom-up). */
int or_reduce(const float* disp, int H, int W, int s, int dmax, int mode, int pixel_grid, int16_t* q)
{
    if (H < 0 || W < 0 || s < 1 || s > 64 || dmax < 1 || dmax > 2047) return OR_E_ARG;
    const int C = W / s;
    int32_t vals[64];
    for (int c = 0; c < C; ++c) {
        for (int r = 0; r < H; ++r) {
            for (int i = 0; i < s; ++i) vals[i] = q4_of(disp[(size_t)r * W + (size_t)c * s + i], dmax);
            int32_t out;
            if (mode == 0) {
                /* lower median: the element of rank floor((s-1)/2) in ascending order (insertion sort) */
                for (int i = 1; i < s; ++i) {
                    int32_t x = vals[i];
                    int j = i - 1;
                    while (j >= 0 && vals[j] > x) { vals[j + 1] = vals[j]; --j; }
                    vals[j + 1] = x;
                }
                out = vals[(s - 1) / 2];
            } else {
                /* mean rounded half up: floor((2 sum + s) / (2 s)) */
                int64_t sum = 0;
                for (int i = 0; i < s; ++i) sum += vals[i];
                out = (int32_t)((2 * sum + s) / (2 * (int64_t)s));
            }
            if (pixel_grid) {
                /* whole pixels (Sec. 3.4 rounds to integer disparities): the nearest
                 * integer to out / 16, halves up, back on the 1/16-px scale */
                const int32_t px = (int32_t)floor((double)out / 16.0 + 0.5);
                out = 16 * px;
            }
            q[(size_t)c * H + (size_t)(H - 1 - r)] = (int16_t)out;
        }
    }
    return OR_OK;
}

/* ------------------------------------------------- ground line from the frame (v-disparity) */

/* The paper takes the ground slope and the horizon as known for every image
 * (Sec. 3); this estimates them from the frame, the step before the path, on
 * the 1/16-px grid the DP uses:
 *   hist[r][e] = number of columns whose reduced code at image row r is e,
 *                for codes e in [16, 16 dmax] (below 1 px: sky / invalid, left out);
 *   S[r][e]    = sum over |t| <= 16 of (17 - |t|) hist[r][e + t]  (a triangular
 *                kernel of half-width 1 px, so noisy ground still votes);
 *   line (k, h): code (k (r - h) + 8) / 16 at image row r > h (the disparity
 *                (k / 256) (r - h) px rounded half up on the 1/16 grid), for
 *                k = 1..256 and every image row h;
 *   votes(k, h) = sum of S[r][code] over the rows r > h whose code lies in
 *                [16, 16 dmax];
 * and returns the line with the most votes, ties to the smaller k, then the
 * smaller h: out = {k, h, votes}.  Lines that are exact on a noise-free ground
 * win strictly: an exact code scores 17 per pixel, a code off by 1/16 px 16. */
int or_ground_estimate(const int16_t* q, int ncols, int H, int dmax, int32_t* out)
{
    if (ncols < 0 || H < 1 || dmax < 1 || !out) return OR_E_ARG;
    const int E = 16 * dmax + 1;
    int64_t* hist = (int64_t*)calloc((size_t)H * E, sizeof(int64_t));
    int64_t* sm = (int64_t*)calloc((size_t)H * E, sizeof(int64_t));
    if (!hist || !sm) { free(hist); free(sm); return OR_E_MEM; }
    for (int c = 0; c < ncols; ++c)
        for (int v = 0; v < H; ++v) {
            const int code = q[(size_t)c * H + v];
            if (code >= 16 && code < E) hist[(size_t)(H - 1 - v) * E + code] += 1;
        }
    for (int r = 0; r < H; ++r)
        for (int e = 16; e < E; ++e) {
            int64_t acc = 0;
            for (int t = -16; t <= 16; ++t) {
                const int x = e + t;
                if (x >= 16 && x < E) acc += (17 - (t < 0 ? -t : t)) * hist[(size_t)r * E + x];
            }
            sm[(size_t)r * E + e] = acc;
        }
    int64_t best = -1;
    int bk = 0, bh = 0;
    for (int k = 1; k <= 256; ++k)
        for (int h = 0; h < H; ++h) {
            int64_t votes = 0;
            for (int r = h + 1; r < H; ++r) {
                const int code = (k * (r - h) + 8) / 16;
                if (code >= E) break;
                if (code >= 16) votes += sm[(size_t)r * E + code];
            }
            if (votes > best) { best = votes; bk = k; bh = h; }
        }
    free(hist);
    free(sm);
    out[0] = bk;
    out[1] = bh;
    out[2] = (int32_t)best;
    return OR_OK;
}

/* --------------------------------------------------------- 2./3. costs and prefix sums */

/* Per-pixel cost of Eq. 4 for one pixel (exposed for tests). */
int or_pixel_cost(const or_params_t* p, int H, int cls, int v, int q, int f, double* out)
{
    or_model_t m;
    int rc = model_build(p, H, &m);
    if (rc) return rc;
    if (cls < 0 || cls > 2 || v < 0 || v >= H || q < 0 || q > 16 * p->dmax || f < 0 || f > p->dmax) {
        model_free(&m);
        return OR_E_ARG;
    }
    *out = pixel_cost(&m, cls, v, q, f);
    model_free(&m);
    return OR_OK;
}

/* Gaussian-branch cost of Eq. 4 at a real disparity d (no min with the outlier
 * branch, no grid) for a model disparity f and class cls; exposed so that tests
 * can check that exp(-cost) integrates to 1 - p_out over [0, d_range]. */
int or_gaussian_branch(const or_params_t* p, int cls, double f, double d, double* out)
{
    int rc = check_params(p);
    if (rc) return rc;
    double base = cls == OR_OBJECT ? p->sigma_object : (cls == OR_GROUND ? p->sigma_ground : p->sigma_sky);
    double sigma = sigma_at(p, base, f);
    *out = k_const(f, sigma, (double)p->p_out, (double)p->dmax) + resid_term(d - f, sigma);
    return OR_OK;
}

/* Model constants (exposed so that tests can compare them with the library's
 * own, independently computed tables).  Costs are in cost units. */
int or_model_constants(const or_params_t* p, int H, double* c_out, double* k_obj /*[dmax+1]*/,
                       double* k_sky, double* fg /*[H]*/, double* k_ground /*[H]*/,
                       double* first /*[3]*/, double* trans /*[9]*/, double* pens /*[3]*/)
{
    or_model_t m;
    int rc = model_build(p, H, &m);
    if (rc) return rc;
    *c_out = maybe_grid(&m, m.c_out);
    for (int f = 0; f <= m.dmax; ++f) k_obj[f] = maybe_grid(&m, m.k_obj[f]);
    *k_sky = maybe_grid(&m, m.k_sky);
    for (int v = 0; v < H; ++v) { fg[v] = m.fg[v]; k_ground[v] = maybe_grid(&m, m.k_ground[v]); }
    for (int c = 0; c < 3; ++c) {
        first[c] = m.first[c];
        for (int q = 0; q < 3; ++q) trans[3 * c + q] = m.trans[c][q];
    }
    pens[0] = m.pen_grav; pens[1] = m.pen_div; pens[2] = m.pen_ord;
    model_free(&m);
    return OR_OK;
}

/* Prefix sums with a leading zero (Sec. 3.4): pd[v+1] = sum of q over rows
 * 0..v; pg, ps likewise for the ground and sky pixel costs; po[f*(H+1) + v+1]
 * for the object cost at integer disparity f. */
static void build_prefix(const or_model_t* m, const int16_t* q, int64_t* pd, double* pg, double* ps, double* po)
{
    const int H = m->H;
    pd[0] = 0; pg[0] = 0.0; ps[0] = 0.0;
    for (int v = 0; v < H; ++v) {
        pd[v + 1] = pd[v] + q[v];
        pg[v + 1] = pg[v] + pixel_cost(m, OR_GROUND, v, q[v], 0);
        ps[v + 1] = ps[v] + pixel_cost(m, OR_SKY, v, q[v], 0);
    }
    for (int f = 0; f <= m->dmax; ++f) {
        double* row = po + (size_t)f * (H + 1);
        row[0] = 0.0;
        for (int v = 0; v < H; ++v) row[v + 1] = row[v] + pixel_cost(m, OR_OBJECT, v, q[v], f);
    }
}

int or_prefix(const or_params_t* p, const int16_t* q, int H, int64_t* pd, double* pg, double* ps, double* po)
{
    or_model_t m;
    int rc = model_build(p, H, &m);
    if (rc) return rc;
    build_prefix(&m, q, pd, pg, ps, po);
    model_free(&m);
    return OR_OK;
}

/* --------------------------------------------------------------- 4./5. the DP */


/* Take candidate (cost, b, p) if it beats the incumbent in (cost, p, b) order.
 * Candidates arrive in ascending b, so an equal (cost, p) never replaces. */
static void consider(double cost, int b, int p, double* best, double* second, int* bb, int* bp)
{
    if (cost < *best || (cost == *best && p < *bp)) {
        *second = *best;
        *best = cost; *bb = b; *bp = p;
    } else if (cost < *second) {
        *second = cost;
    }
}

typedef struct {
    double cost;        /* minimum total cost of the column */
    double gap_abs;     /* min over the backtracked path of (runner-up - best) */
    double gap_rel;     /* min over the path of (runner-up - best) / max(1, |best|) */
    int32_t n;          /* number of stixels on the path (may exceed the capacity) */
} or_column_result_t;

static int column_dp(const or_model_t* m, const int16_t* q, int cap, or_stixel_t* out, or_column_result_t* res)
{
    const int H = m->H, F = m->dmax + 1;
    int64_t* pd = (int64_t*)malloc(sizeof(int64_t) * (size_t)(H + 1));
    double* pg = (double*)malloc(sizeof(double) * (size_t)(H + 1));
    double* ps = (double*)malloc(sizeof(double) * (size_t)(H + 1));
    double* po = (double*)malloc(sizeof(double) * (size_t)F * (H + 1));
    double* V = (double*)malloc(sizeof(double) * 3 * (size_t)H);       /* cost table */
    double* G = (double*)malloc(sizeof(double) * 3 * (size_t)H);       /* runner-up per cell */
    int32_t* BB = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)H);   /* index table: start row */
    int32_t* BP = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)H);   /* index table: previous class */
    int32_t* fob = (int32_t*)malloc(sizeof(int32_t) * (size_t)H);      /* f of ob^k */
    or_stixel_t* path = (or_stixel_t*)malloc(sizeof(or_stixel_t) * (size_t)H);
    if (!pd || !pg || !ps || !po || !V || !G || !BB || !BP || !fob || !path) {
        free(pd); free(pg); free(ps); free(po); free(V); free(G); free(BB); free(BP); free(fob); free(path);
        return OR_E_MEM;
    }
    build_prefix(m, q, pd, pg, ps, po);

    for (int k = 0; k < H; ++k) {
        for (int c = 0; c < 3; ++c) {
            double best = INFINITY, second = INFINITY;
            int bb = -1, bp = OR_NONE + 1;
            for (int b = 0; b <= k; ++b) {
                const int n = k - b + 1;
                const int64_t S = pd[k + 1] - pd[b];
                const int f = mean_f(S, n);
                double data;
                if (c == OR_OBJECT) data = po[(size_t)f * (H + 1) + k + 1] - po[(size_t)f * (H + 1) + b];
                else if (c == OR_GROUND) data = pg[k + 1] - pg[b];
                else data = ps[k + 1] - ps[b];
                if (b == 0) {                       /* Eq. 5 / first row of Eq. 6 */
                    consider(data + m->first[c], 0, OR_NONE, &best, &second, &bb, &bp);
                } else {
                    for (int p = 0; p < 3; ++p) {
                        double prev = V[3 * (b - 1) + p];
                        double cand = data + pair_prior(m, c, p, b, f, fob[b - 1]) + prev;
                        consider(cand, b, p, &best, &second, &bb, &bp);
                    }
                }
            }
            V[3 * k + c] = best;
            G[3 * k + c] = second;
            BB[3 * k + c] = bb;
            BP[3 * k + c] = bp;
            if (c == OR_OBJECT) fob[k] = bb >= 0 ? mean_f(pd[k + 1] - pd[bb], k - bb + 1) : 0;
        }
    }

    /* top row: C_min = min(OB, GR, SK) in the order object < ground < sky */
    int c = OR_OBJECT;
    for (int cc = 1; cc < 3; ++cc)
        if (V[3 * (H - 1) + cc] < V[3 * (H - 1) + c]) c = cc;
    double top_second = INFINITY;   /* smallest of the two classes not chosen */
    for (int cc = 0; cc < 3; ++cc)
        if (cc != c && V[3 * (H - 1) + cc] < top_second) top_second = V[3 * (H - 1) + cc];
    res->cost = V[3 * (H - 1) + c];
    if (isinf(res->cost)) {
        res->n = 0;
        res->gap_abs = res->gap_rel = 0.0;
        free(pd); free(pg); free(ps); free(po); free(V); free(G); free(BB); free(BP); free(fob); free(path);
        return OR_E_INFEASIBLE;
    }
    double gap_abs = top_second - res->cost;
    double gap_rel = gap_abs / fmax(1.0, fabs(res->cost));

    int n = 0, k = H - 1;
    while (k >= 0) {
        int b = BB[3 * k + c], p = BP[3 * k + c];
        double best = V[3 * k + c], g = G[3 * k + c] - best;
        if (g < gap_abs) gap_abs = g;
        if (g / fmax(1.0, fabs(best)) < gap_rel) gap_rel = g / fmax(1.0, fabs(best));
        or_stixel_t st;
        st.v_bottom = b; st.v_top = k; st.cls = c;
        st.sum_q = pd[k + 1] - pd[b];
        st.f = mean_f(st.sum_q, k - b + 1);
        st.disparity = (double)st.sum_q / (16.0 * (double)(k - b + 1));
        path[n++] = st;
        k = b - 1;
        c = p;
    }
    /* emit bottom -> top */
    for (int i = 0; i < n && i < cap; ++i) out[i] = path[n - 1 - i];
    res->n = n;
    res->gap_abs = gap_abs;
    res->gap_rel = gap_rel;
    free(pd); free(pg); free(ps); free(po); free(V); free(G); free(BB); free(BP); free(fob); free(path);
    return n > cap ? OR_E_CAPACITY : OR_OK;
}

/* Lexicographic order of candidates in the global-MAP DP: cost, then the
 * previous class (object < ground < sky < none), start row, previous object f. */
typedef struct { double cost; int p, b, fprev; } map_key_t;

static int key_less(map_key_t a, map_key_t b)
{
    if (a.cost != b.cost) return a.cost < b.cost;
    if (a.p != b.p) return a.p < b.p;
    if (a.b != b.b) return a.b < b.b;
    return a.fprev < b.fprev;
}

/* The global MAP (global_map = 1): states (row k, object, f) for every mean
 * disparity f of the top stixel, and (row k, ground), (row k, sky); a stixel
 * [b, k] of class c extends every state of row b - 1 with the exact prior of
 * the pair (for object above object: the ordering penalty against that
 * state's f).  Evaluated plainly: every end row, start row, previous class and
 * previous object disparity.  gap_abs / gap_rel are not computed (0). */
static int column_dp_map(const or_model_t* m, const int16_t* q, int cap, or_stixel_t* out, or_column_result_t* res)
{
    const int H = m->H, F = m->dmax + 1;
    const size_t NO = (size_t)H * F;
    int64_t* pd = (int64_t*)malloc(sizeof(int64_t) * (size_t)(H + 1));
    double* pg = (double*)malloc(sizeof(double) * (size_t)(H + 1));
    double* ps = (double*)malloc(sizeof(double) * (size_t)(H + 1));
    double* po = (double*)malloc(sizeof(double) * (size_t)F * (H + 1));
    map_key_t* KO = (map_key_t*)malloc(sizeof(map_key_t) * NO);          /* [k][f] object states */
    map_key_t* KG = (map_key_t*)malloc(sizeof(map_key_t) * (size_t)H);    /* ground states */
    map_key_t* KS = (map_key_t*)malloc(sizeof(map_key_t) * (size_t)H);    /* sky states */
    or_stixel_t* path = (or_stixel_t*)malloc(sizeof(or_stixel_t) * (size_t)H);
    if (!pd || !pg || !ps || !po || !KO || !KG || !KS || !path) {
        free(pd); free(pg); free(ps); free(po); free(KO); free(KG); free(KS); free(path);
        return OR_E_MEM;
    }
    build_prefix(m, q, pd, pg, ps, po);
    const map_key_t none = {INFINITY, OR_NONE, 0, 0};

    for (int k = 0; k < H; ++k) {
        for (int f = 0; f < F; ++f) KO[(size_t)k * F + f] = none;
        KG[k] = none;
        KS[k] = none;
        for (int b = 0; b <= k; ++b) {
            const int n = k - b + 1;
            const int64_t S = pd[k + 1] - pd[b];
            const int fo = mean_f(S, n);
            const double data[3] = {po[(size_t)fo * (H + 1) + k + 1] - po[(size_t)fo * (H + 1) + b],
                                    pg[k + 1] - pg[b], ps[k + 1] - ps[b]};
            map_key_t* dst[3] = {&KO[(size_t)k * F + fo], &KG[k], &KS[k]};
            for (int c = 0; c < 3; ++c) {
                if (b == 0) {
                    map_key_t cand = {data[c] + m->first[c], OR_NONE, 0, 0};
                    if (key_less(cand, *dst[c])) *dst[c] = cand;
                    continue;
                }
                for (int fp = 0; fp < F; ++fp) {          /* previous state: object with f = fp */
                    const double prev = KO[(size_t)(b - 1) * F + fp].cost;
                    if (isinf(prev)) continue;
                    map_key_t cand = {data[c] + pair_prior(m, c, OR_OBJECT, b, fo, fp) + prev, OR_OBJECT, b, fp};
                    if (key_less(cand, *dst[c])) *dst[c] = cand;
                }
                map_key_t cg = {data[c] + pair_prior(m, c, OR_GROUND, b, fo, 0) + KG[b - 1].cost, OR_GROUND, b, 0};
                if (key_less(cg, *dst[c])) *dst[c] = cg;
                map_key_t cs = {data[c] + pair_prior(m, c, OR_SKY, b, fo, 0) + KS[b - 1].cost, OR_SKY, b, 0};
                if (key_less(cs, *dst[c])) *dst[c] = cs;
            }
        }
    }

    /* top row: lexicographic (cost, class, f), classes object < ground < sky */
    int c = -1, f = 0;
    double best = INFINITY;
    for (int ff = 0; ff < F; ++ff)
        if (KO[(size_t)(H - 1) * F + ff].cost < best) { best = KO[(size_t)(H - 1) * F + ff].cost; c = OR_OBJECT; f = ff; }
    if (KG[H - 1].cost < best) { best = KG[H - 1].cost; c = OR_GROUND; f = 0; }
    if (KS[H - 1].cost < best) { best = KS[H - 1].cost; c = OR_SKY; f = 0; }
    res->cost = best;
    res->gap_abs = res->gap_rel = 0.0;
    if (c < 0 || isinf(best)) {
        res->n = 0;
        free(pd); free(pg); free(ps); free(po); free(KO); free(KG); free(KS); free(path);
        return OR_E_INFEASIBLE;
    }
    int n = 0, k = H - 1;
    while (k >= 0 && c != OR_NONE) {
        const map_key_t key = c == OR_OBJECT ? KO[(size_t)k * F + f] : (c == OR_GROUND ? KG[k] : KS[k]);
        const int b = key.b;
        or_stixel_t st;
        st.v_bottom = b; st.v_top = k; st.cls = c;
        st.sum_q = pd[k + 1] - pd[b];
        st.f = mean_f(st.sum_q, k - b + 1);
        st.disparity = (double)st.sum_q / (16.0 * (double)(k - b + 1));
        path[n++] = st;
        k = b - 1;
        c = key.p;
        f = key.fprev;
    }
    for (int i = 0; i < n && i < cap; ++i) out[i] = path[n - 1 - i];
    res->n = n;
    free(pd); free(pg); free(ps); free(po); free(KO); free(KG); free(KS); free(path);
    return n > cap ? OR_E_CAPACITY : OR_OK;
}

/* One column: q[0..H-1] bottom-up Q4 codes.  Writes up to cap stixels. */
int or_column(const or_params_t* p, const int16_t* q, int H, int cap, or_stixel_t* out, or_column_result_t* res)
{
    or_model_t m;
    int rc = model_build(p, H, &m);
    if (rc) return rc;
    rc = p->global_map ? column_dp_map(&m, q, cap, out, res) : column_dp(&m, q, cap, out, res);
    model_free(&m);
    return rc;
}

/* A whole frame: reduction then every column (columns in parallel when the
 * library is built with OpenMP; nthreads <= 0 uses the default team).
 * out: ncols x cap stixels; res: ncols results; q (optional): ncols x H. */
int or_frame(const or_params_t* p, const float* disp, int H, int W, int cap, or_stixel_t* out,
             or_column_result_t* res, int16_t* q_out, int nthreads)
{
    const int s = p->stixel_width;
    if (s < 1 || H < 1 || W < 0 || cap < 0) return OR_E_ARG;
    const int C = W / s;
    int16_t* q = q_out ? q_out : (int16_t*)malloc(sizeof(int16_t) * (size_t)C * H + 1);
    if (!q) return OR_E_MEM;
    int rc = or_reduce(disp, H, W, s, p->dmax, p->reduce_mode, p->pixel_grid, q);
    if (rc) { if (!q_out) free(q); return rc; }
    int32_t line[3] = {0, 0, 0};
    if (p->ground_estimate) {
        rc = or_ground_estimate(q, C, H, p->dmax, line);
        if (rc) { if (!q_out) free(q); return rc; }
        if (line[2] == 0) line[0] = 0;          /* no ground seen: keep the camera's line */
    }
    or_model_t m;
    rc = model_build_line(p, H, line[0], line[1], &m);
    if (rc) { if (!q_out) free(q); return rc; }
    int worst = OR_OK;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int c = 0; c < C; ++c) {
        int r = p->global_map ? column_dp_map(&m, q + (size_t)c * H, cap, out + (size_t)c * cap, res + c)
                              : column_dp(&m, q + (size_t)c * H, cap, out + (size_t)c * cap, res + c);
        if (r != OR_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
            { if (worst == OR_OK || r != OR_E_CAPACITY) worst = r; }
        }
    }
    (void)nthreads;
    model_free(&m);
    if (!q_out) free(q);
    return worst;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------- direct evaluation and brute force */

/* Cost of one stixel's data term as a direct per-pixel sum (no prefix sums). */
static double direct_data(const or_model_t* m, const int16_t* q, int c, int b, int k, int f)
{
    double s = 0.0;
    for (int v = b; v <= k; ++v) s += pixel_cost(m, c, v, q[v], f);
    return s;
}

/* Total cost of a given segmentation (bottom -> top list of n stixels, bounds
 * and classes only), from direct per-pixel sums and the true priors of each
 * adjacent pair.  Returns INFINITY for an invalid list (gaps, overlaps, bad
 * class) -- callers check validity separately. */
/* The total of a segmentation under model m (see or_eval_segmentation). */
static double eval_with_model(const or_model_t* m, const int16_t* q, const or_stixel_t* st, int n)
{
    const int H = m->H;
    double total = 0.0;
    int prev_c = OR_NONE, prev_f = 0, expect_b = 0;
    for (int i = 0; i < n; ++i) {
        int b = st[i].v_bottom, k = st[i].v_top, c = st[i].cls;
        if (b != expect_b || k < b || k >= H || c < 0 || c > 2) return INFINITY;
        int64_t S = 0;
        for (int v = b; v <= k; ++v) S += q[v];
        int f = mean_f(S, k - b + 1);
        total += direct_data(m, q, c, b, k, f);
        total += (i == 0) ? m->first[c] : pair_prior(m, c, prev_c, b, f, prev_f);
        prev_c = c; prev_f = f; expect_b = k + 1;
    }
    return expect_b == H ? total : INFINITY;
}

int or_eval_segmentation(const or_params_t* p, const int16_t* q, int H, const or_stixel_t* st, int n, double* out)
{
    or_model_t m;
    int rc = model_build(p, H, &m);
    if (rc) return rc;
    *out = eval_with_model(&m, q, st, n);
    model_free(&m);
    return OR_OK;
}

/* The totals of one segmentation per column of a frame's reduced codes q
 * (ncols x H, bottom-up), under the frame's model: the camera's ground line,
 * or with ground_estimate the line or_frame estimates from the same codes.
 * st: ncols x cap stixels, counts[c] of them used (a column with
 * counts[c] > cap gets NaN: its list is incomplete). */
int or_eval_frame(const or_params_t* p, const int16_t* q, int ncols, int H, const or_stixel_t* st, int cap,
                  const int32_t* counts, double* out)
{
    if (ncols < 0 || H < 1 || cap < 0) return OR_E_ARG;
    int32_t line[3] = {0, 0, 0};
    if (p->ground_estimate) {
        int rc = or_ground_estimate(q, ncols, H, p->dmax, line);
        if (rc) return rc;
        if (line[2] == 0) line[0] = 0;          /* no ground seen: the camera's line */
    }
    or_model_t m;
    int rc = model_build_line(p, H, line[0], line[1], &m);
    if (rc) return rc;
    for (int c = 0; c < ncols; ++c)
        out[c] = counts[c] > cap ? NAN
                                 : eval_with_model(&m, q + (size_t)c * H, st + (size_t)c * cap, counts[c]);
    model_free(&m);
    return OR_OK;
}

/* Enumerate every segmentation of a column with H <= 14 rows: all 2^(H-1) cut
 * patterns times all 3^N class labellings.  Returns the minimum cost, how many
 * segmentations reach it, and the first one reached in enumeration order
 * (cut mask ascending, then labels as base-3 digits bottom stixel first). */
int or_brute_force(const or_params_t* p, const int16_t* q, int H, double* best_cost, int64_t* n_best,
                   or_stixel_t* out, int32_t* n_out)
{
    if (H < 1 || H > 14) return OR_E_ARG;
    or_model_t m;
    int rc = model_build(p, H, &m);
    if (rc) return rc;
    /* data cost of every (class, b, k) by direct sums, and the rounded means */
    double data[3][14][14];
    int fm[14][14];
    for (int b = 0; b < H; ++b)
        for (int k = b; k < H; ++k) {
            int64_t S = 0;
            for (int v = b; v <= k; ++v) S += q[v];
            fm[b][k] = mean_f(S, k - b + 1);
            for (int c = 0; c < 3; ++c) data[c][b][k] = direct_data(&m, q, c, b, k, fm[b][k]);
        }
    double best = INFINITY;
    int64_t count = 0;
    int bestN = 0, bestB[14], bestK[14], bestC[14];
    const uint32_t masks = 1u << (H - 1);
    for (uint32_t mask = 0; mask < masks; ++mask) {
        int N = 0, B[14], K[14];
        int start = 0;
        for (int i = 0; i < H - 1; ++i)
            if (mask & (1u << i)) { B[N] = start; K[N] = i; ++N; start = i + 1; }
        B[N] = start; K[N] = H - 1; ++N;
        int lab[14] = {0};
        for (;;) {
            double cost = 0.0;
            for (int i = 0; i < N && cost < INFINITY; ++i) {
                int c = lab[i];
                cost += data[c][B[i]][K[i]];
                if (i == 0) cost += m.first[c];
                else cost += pair_prior(&m, c, lab[i - 1], B[i], fm[B[i]][K[i]], fm[B[i - 1]][K[i - 1]]);
            }
            if (cost < best) {
                best = cost; count = 1; bestN = N;
                for (int i = 0; i < N; ++i) { bestB[i] = B[i]; bestK[i] = K[i]; bestC[i] = lab[i]; }
            } else if (cost == best && cost < INFINITY) {
                ++count;
            }
            int i = 0;
            while (i < N && lab[i] == 2) lab[i++] = 0;
            if (i == N) break;
            ++lab[i];
        }
    }
    *best_cost = best;
    *n_best = count;
    *n_out = bestN;
    for (int i = 0; i < bestN; ++i) {
        int64_t S = 0;
        for (int v = bestB[i]; v <= bestK[i]; ++v) S += q[v];
        out[i].v_bottom = bestB[i]; out[i].v_top = bestK[i]; out[i].cls = bestC[i];
        out[i].sum_q = S; out[i].f = mean_f(S, bestK[i] - bestB[i] + 1);
        out[i].disparity = (double)S / (16.0 * (double)(bestK[i] - bestB[i] + 1));
    }
    model_free(&m);
    return OR_OK;
}
