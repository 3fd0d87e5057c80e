/*
 * FP64 CPU oracle for differentiable 2D Gaussian ray tracing (IRGS,
 * arXiv 2412.15867) -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, brute-force definition that the CUDA tracer is
 * checked against. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it. It shares no code, header or constant table
 * with the CUDA library; the two only consume the same float32 input arrays.
 *
 * What it computes (paper sections cited per function):
 *   - oracle_trace:  every ray against every surfel (Eq. 6-7), hits sorted by
 *                    (tau, user index), alpha-blended front to back (Eq. 2, 8)
 *                    with early termination on transmittance (Sec. 4 impl.).
 *   - oracle_trace_grad: the analytic gradient of the blended outputs with
 *                    respect to every surfel parameter (the tracer is
 *                    differentiable, Sec. 3.3, light parametrization),
 *                    accumulating the suffix sum with a reverse loop.
 *   - oracle_shade:  the Monte Carlo rendering-equation estimate of Eq. 15
 *                    with Eq. 13-14 light decomposition, using cosine and GGX
 *                    importance sampling (supplementary "Composited scene").
 *
 * Readings where the paper is silent (all shared with the CUDA side through
 * the parameters only, never through code):
 *   - support cut rho^2 <= rho_c^2, rho_c = min(3, sqrt(2 ln(o/alpha_min)));
 *     alpha = min(alpha_max, o exp(-rho^2/2)); rejected if alpha < alpha_min;
 *   - a hit needs t_min < tau < t_max; |n.d| < 1e-8 |d| is no hit;
 *   - termination: the hit that makes T < T_min is included, then stop;
 *   - quaternion (w,x,y,z), normalised here; rotation columns (t_u, t_v, n);
 *   - BRDF: GGX D with alpha_g = r^2, Schlick F (F0 = 0.04) on (w_o.h),
 *     separable Schlick-GGX G with k = alpha_g/2, f_d = a/pi;
 *   - random numbers: SplitMix64 (Steele, Lea, Flood 2014) stream outputs,
 *     top 24 bits -> [0,1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

typedef struct {
    double alpha_min;   /* alpha cutoff (also sets the support radius)   */
    double alpha_max;   /* alpha clamp                                  */
    double T_min;       /* stop once transmittance falls below this     */
    double t_min;       /* hits need tau > t_min                        */
    double t_max;       /* hits need tau < t_max                        */
    int32_t feat_offset;/* first blended feature channel                */
    int32_t feat_count; /* number of blended feature channels           */
} oracle_params;

/* Per-ray ambiguity flags: a ray is flagged when the exact answer sits within
 * a margin of a discontinuity, so that a correct FP32 implementation may land
 * on either side. */
typedef struct {
    double alpha_abs;   /* |alpha_raw - alpha_min| < alpha_abs             */
    double rho_rel;     /* |rho^2 - rho_c^2| < rho_rel * rho_c^2           */
    double T_rel;       /* |T - T_min| < T_rel * T_min after a hit         */
    double tie_abs;     /* |tau_j - tau_j+1| < tie_abs * max(1, tau)       */
    double t_abs;       /* |tau - t_min| or |tau - t_max| < t_abs          */
    double clamp_abs;   /* |alpha_raw - alpha_max| < clamp_abs (gradients) */
} oracle_margins;

enum {
    OF_ALPHA = 1u, OF_RHO = 2u, OF_T = 4u, OF_TIE = 8u, OF_TRANGE = 16u,
    OF_GRAZE = 32u, OF_CLAMP = 64u
};

/* ---------------------------------------------------------------------- */
/* Surfel geometry in FP64 (Sec. 3.2: centre mu, tangents t_u, t_v, scales  */
/* s_u, s_v, normal n = t_u x t_v; Sec. 3.1: rotation from a quaternion).  */
/* ---------------------------------------------------------------------- */
typedef struct {
    double mu[3], tu[3], tv[3], n[3];
    double su, sv, o, rc2;   /* rc2 < 0: never hit */
    double q[4], qn;         /* raw quaternion and its norm (for gradients) */
} surfel64;

/* Rotation matrix of the unit quaternion (w,x,y,z); returns its columns. */
static void quat_frame(const double qh[4], double tu[3], double tv[3], double n[3])
{
    double w = qh[0], x = qh[1], y = qh[2], z = qh[3];
    tu[0] = 1.0 - 2.0 * (y * y + z * z); tu[1] = 2.0 * (x * y + w * z); tu[2] = 2.0 * (x * z - w * y);
    tv[0] = 2.0 * (x * y - w * z); tv[1] = 1.0 - 2.0 * (x * x + z * z); tv[2] = 2.0 * (y * z + w * x);
    n[0]  = 2.0 * (x * z + w * y); n[1]  = 2.0 * (y * z - w * x); n[2]  = 1.0 - 2.0 * (x * x + y * y);
}

static void load_surfels(const float* means, const float* quats, const float* scales,
                         const float* opacity, int64_t n, double alpha_min, surfel64* s)
{
    for (int64_t i = 0; i < n; ++i) {
        surfel64* S = &s[i];
        double q[4];
        for (int k = 0; k < 4; ++k) q[k] = (double)quats[4 * i + k];
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double qh[4] = {q[0] / qn, q[1] / qn, q[2] / qn, q[3] / qn};
        quat_frame(qh, S->tu, S->tv, S->n);
        for (int k = 0; k < 3; ++k) S->mu[k] = (double)means[3 * i + k];
        for (int k = 0; k < 4; ++k) S->q[k] = q[k];
        S->qn = qn;
        S->su = (double)scales[2 * i];
        S->sv = (double)scales[2 * i + 1];
        S->o = (double)opacity[i];
        /* Eq. 5 support radius sqrt(2 ln(o/alpha_min)), capped at 3 sigma */
        if (S->o > 0.0) {
            double r2 = 2.0 * log(S->o / alpha_min);
            S->rc2 = r2 < 9.0 ? r2 : 9.0;
        } else {
            S->rc2 = -1.0;
        }
    }
}

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* One ray-surfel candidate (Eq. 6-7). */
typedef struct {
    double tau, u, v, rho2, G, alpha_raw, alpha, den;
    double e[3];      /* p - mu */
    int64_t id;
} cand64;

/* Returns 1 if the ray meets the surfel's plane (non-grazing) and fills c. */
static int intersect(const surfel64* S, const double o[3], const double d[3], cand64* c)
{
    double dn = sqrt(dot3(d, d));
    double den = dot3(S->n, d);
    c->den = den;
    if (den == 0.0) return 0;
    double mo[3] = {S->mu[0] - o[0], S->mu[1] - o[1], S->mu[2] - o[2]};
    double tau = dot3(S->n, mo) / den;                    /* Eq. 6 */
    double p[3] = {o[0] + tau * d[0], o[1] + tau * d[1], o[2] + tau * d[2]};
    for (int k = 0; k < 3; ++k) c->e[k] = p[k] - S->mu[k];
    c->tau = tau;
    c->u = dot3(c->e, S->tu) / S->su;                      /* Eq. 7 */
    c->v = dot3(c->e, S->tv) / S->sv;
    c->rho2 = c->u * c->u + c->v * c->v;
    c->G = exp(-0.5 * c->rho2);
    c->alpha_raw = S->o * c->G;
    return fabs(den) >= 1e-8 * dn;   /* grazing rays do not hit */
}

typedef struct { double tau, alpha; int64_t id; } hit64;

static int hit_cmp(const void* a, const void* b)
{
    const hit64* x = (const hit64*)a;
    const hit64* y = (const hit64*)b;
    if (x->tau < y->tau) return -1;
    if (x->tau > y->tau) return 1;
    return (x->id < y->id) ? -1 : (x->id > y->id);
}

/* Ray march of one ray: collect all hits, sort by (tau, id), and return the
 * number of hits kept in `hits` (capacity n). Sets *flags if non-NULL using
 * the margins (only candidates before the termination point matter, which
 * the caller resolves after compositing). */
typedef struct { double tau; uint32_t kind; } near64;

static int64_t collect_hits(const surfel64* s, int64_t n, const double o[3], const double d[3],
                            const oracle_params* P, const oracle_margins* M,
                            hit64* hits, near64* nears, int64_t* n_near)
{
    int64_t nh = 0, nn = 0;
    double dn = sqrt(dot3(d, d));
    for (int64_t i = 0; i < n; ++i) {
        const surfel64* S = &s[i];
        cand64 c;
        if (S->rc2 < 0.0) continue;
        if (!intersect(S, o, d, &c)) {
            /* grazing, but close enough to the threshold that it might count */
            if (M && c.den != 0.0 && fabs(c.den) >= 0.5e-8 * dn && c.rho2 <= S->rc2 * (1.0 + M->rho_rel)
                && c.alpha_raw >= P->alpha_min - M->alpha_abs) {
                nears[nn].tau = c.tau; nears[nn].kind = OF_GRAZE; nn++;
            }
            continue;
        }
        uint32_t kind = 0;
        if (M) {
            if (fabs(c.rho2 - S->rc2) < M->rho_rel * (S->rc2 > 1e-12 ? S->rc2 : 1e-12)) kind |= OF_RHO;
            if (fabs(c.alpha_raw - P->alpha_min) < M->alpha_abs) kind |= OF_ALPHA;
            if (fabs(c.tau - P->t_min) < M->t_abs || (isfinite(P->t_max) && fabs(c.tau - P->t_max) < M->t_abs))
                kind |= OF_TRANGE;
            if (fabs(c.alpha_raw - P->alpha_max) < M->clamp_abs) kind |= OF_CLAMP;
            if (fabs(c.den) < 2e-8 * dn) kind |= OF_GRAZE;
        }
        int accepted = 1;
        if (c.rho2 > S->rc2) accepted = 0;
        double alpha = c.alpha_raw < P->alpha_max ? c.alpha_raw : P->alpha_max;
        if (alpha < P->alpha_min) accepted = 0;
        if (!(c.tau > P->t_min && c.tau < P->t_max)) accepted = 0;
        if (kind && (accepted || (kind & (OF_RHO | OF_ALPHA | OF_TRANGE | OF_GRAZE)))) {
            nears[nn].tau = c.tau; nears[nn].kind = kind; nn++;
        }
        if (!accepted) continue;
        hits[nh].tau = c.tau;
        hits[nh].alpha = alpha;
        hits[nh].id = i;
        nh++;
    }
    qsort(hits, (size_t)nh, sizeof(hit64), hit_cmp);
    if (n_near) *n_near = nn;
    return nh;
}

/* Front-to-back blending of the sorted hits (Eq. 2 and Eq. 8; Eq. 9 weights
 * unnormalised). Returns the number of composited hits. */
static int64_t composite(const hit64* hits, int64_t nh, const float* feats, int32_t F_total,
                         const oracle_params* P, double* C, double* D, double* Tfin,
                         double* Tlist /* transmittance before each hit, or NULL */)
{
    double T = 1.0;
    for (int c = 0; c < P->feat_count; ++c) C[c] = 0.0;
    *D = 0.0;
    int64_t j = 0;
    for (; j < nh; ++j) {
        if (Tlist) Tlist[j] = T;
        double w = T * hits[j].alpha;
        const float* f = feats ? feats + hits[j].id * (int64_t)F_total + P->feat_offset : NULL;
        for (int c = 0; c < P->feat_count; ++c) C[c] += w * (double)f[c];
        *D += w * hits[j].tau;
        T *= (1.0 - hits[j].alpha);
        if (T < P->T_min) { ++j; break; }
    }
    *Tfin = T;
    return j;
}

static uint32_t resolve_flags(const hit64* hits, int64_t nh, int64_t ncomp, const near64* nears,
                              int64_t nn, const oracle_params* P, const oracle_margins* M,
                              const double* Tlist, double Tfin)
{
    uint32_t f = 0;
    /* candidates beyond the termination point cannot matter */
    double tau_stop = (ncomp < nh || (ncomp > 0 && Tfin < P->T_min)) && ncomp > 0
                          ? hits[ncomp - 1].tau : INFINITY;
    for (int64_t i = 0; i < nn; ++i) {
        double lim = tau_stop + M->tie_abs * (fabs(tau_stop) > 1.0 ? fabs(tau_stop) : 1.0);
        if (nears[i].tau <= lim) f |= nears[i].kind;
    }
    /* near-equal depths among the composited hits and the next one */
    int64_t last = ncomp < nh ? ncomp : nh - 1;
    for (int64_t j = 0; j < last; ++j) {
        double t = fabs(hits[j].tau) > 1.0 ? fabs(hits[j].tau) : 1.0;
        if (fabs(hits[j + 1].tau - hits[j].tau) < M->tie_abs * t) f |= OF_TIE;
    }
    /* transmittance close to the threshold after any composited hit */
    for (int64_t j = 0; j < ncomp; ++j) {
        double Tafter = (j + 1 < ncomp) ? Tlist[j + 1] : Tfin;
        if (fabs(Tafter - P->T_min) < M->T_rel * P->T_min) f |= OF_T;
    }
    return f;
}

static int nthreads_set(int n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
    return omp_get_max_threads();
#else
    (void)n_threads;
    return 1;
#endif
}

int oracle_num_threads(int n_threads) { return nthreads_set(n_threads); }

/* Forward trace of R rays (Eq. 8). Outputs: feat [R, feat_count], depth [R]
 * (sum of w tau, tau in units of |d|), opacity [R] = 1 - T_final, n_hits [R];
 * optionally the composited user ids and depths [R, max_ids] (-1 / NaN
 * padded) and the ambiguity flags [R]. Returns 0, or -1 on bad arguments. */
int oracle_trace(const float* means, const float* quats, const float* scales, const float* opacity,
                 const float* feats, int64_t n, int32_t F_total,
                 const float* ray_o, const float* ray_d, int64_t R,
                 const oracle_params* P, const oracle_margins* M,
                 double* out_feat, double* out_depth, double* out_opacity, int32_t* out_nhits,
                 int32_t* out_ids, double* out_tau, int32_t max_ids, uint32_t* out_flags,
                 int n_threads)
{
    if (n < 0 || R < 0 || !P) return -1;
    if (P->feat_count > 0 && (P->feat_offset < 0 || P->feat_offset + P->feat_count > F_total)) return -1;
    surfel64* s = (surfel64*)malloc(sizeof(surfel64) * (size_t)(n > 0 ? n : 1));
    if (!s) return -1;
    load_surfels(means, quats, scales, opacity, n, P->alpha_min, s);
    nthreads_set(n_threads);
    int err = 0;
#pragma omp parallel
    {
        hit64* hits = (hit64*)malloc(sizeof(hit64) * (size_t)(n > 0 ? n : 1));
        near64* nears = (near64*)malloc(sizeof(near64) * (size_t)(n > 0 ? n : 1));
        double* Tl = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        double* C = (double*)malloc(sizeof(double) * (size_t)(P->feat_count > 0 ? P->feat_count : 1));
        if (!hits || !nears || !Tl || !C) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t r = 0; r < R; ++r) {
                double o[3] = {ray_o[3 * r], ray_o[3 * r + 1], ray_o[3 * r + 2]};
                double d[3] = {ray_d[3 * r], ray_d[3 * r + 1], ray_d[3 * r + 2]};
                int64_t nn = 0;
                int64_t nh = collect_hits(s, n, o, d, P, M, hits, nears, &nn);
                double D, Tfin;
                int64_t nc = composite(hits, nh, feats, F_total, P, C, &D, &Tfin, Tl);
                for (int c = 0; c < P->feat_count; ++c) out_feat[r * P->feat_count + c] = C[c];
                out_depth[r] = D;
                out_opacity[r] = 1.0 - Tfin;
                if (out_nhits) out_nhits[r] = (int32_t)nc;
                if (out_ids || out_tau) {
                    for (int32_t j = 0; j < max_ids; ++j) {
                        if (out_ids) out_ids[r * max_ids + j] = j < nc ? (int32_t)hits[j].id : -1;
                        if (out_tau) out_tau[r * max_ids + j] = j < nc ? hits[j].tau : NAN;
                    }
                }
                if (out_flags) out_flags[r] = M ? resolve_flags(hits, nh, nc, nears, nn, P, M, Tl, Tfin) : 0u;
            }
        }
        free(hits); free(nears); free(Tl); free(C);
    }
    free(s);
    return err ? -1 : 0;
}

/* ---------------------------------------------------------------------- */
/* Admissible outcomes of a ray whose exact answer lies within a margin of  */
/* a discontinuity. A correct FP32 tracer may decide such a candidate, such */
/* an order or such a stop either way; every outcome those decisions give   */
/* is composited here by the plain definition (Eq. 2, Eq. 8):               */
/*   - a candidate within a margin of the alpha cutoff, the support edge,   */
/*     an end of the ray interval or the grazing threshold is in or out;    */
/*   - a run of hits whose successive depths differ by less than the tie    */
/*     margin is blended in any order;                                      */
/*   - where the transmittance after a hit lies within T_rel of T_min, the  */
/*     march stops there or goes on (the threshold moved by 2 T_rel).       */
/* Candidates beyond the farthest possible stop (all optional candidates    */
/* out, the lower threshold) cannot change the result and are dropped.     */
/* ---------------------------------------------------------------------- */
typedef struct { double tau, alpha; int64_t id; int optional, def_in; } alt64;

static int alt_cmp(const void* a, const void* b)
{
    const alt64* x = (const alt64*)a;
    const alt64* y = (const alt64*)b;
    if (x->tau < y->tau) return -1;
    if (x->tau > y->tau) return 1;
    return (x->id < y->id) ? -1 : (x->id > y->id);
}

/* Blend the listed entries (order[] indexes L; entries with use[] == 0 are
 * skipped) until T < Tstop. *near_T is set when T after a blended hit lies
 * within T_rel of T_min. Returns the number of blended hits. */
static int64_t alt_composite(const alt64* L, const int64_t* order, const unsigned char* use, int64_t n,
                             const float* feats, int32_t F_total, const oracle_params* P, double Tstop,
                             double T_rel, double* C, double* D, double* Tfin, int* near_T)
{
    double T = 1.0;
    int64_t nc = 0;
    for (int c = 0; c < P->feat_count; ++c) C[c] = 0.0;
    *D = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const alt64* h = &L[order[i]];
        if (!use[order[i]]) continue;
        double w = T * h->alpha;
        const float* f = feats ? feats + h->id * (int64_t)F_total + P->feat_offset : NULL;
        for (int c = 0; c < P->feat_count; ++c) C[c] += w * (double)f[c];
        *D += w * h->tau;
        T *= (1.0 - h->alpha);
        ++nc;
        if (near_T && fabs(T - P->T_min) < T_rel * P->T_min) *near_T = 1;
        if (T < Tstop) break;
    }
    *Tfin = T;
    return nc;
}

static double factorial_d(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return f;
}

/* Work arrays of ray_alternatives (capacity n each, plus one row of C). */
typedef struct { alt64* L; int64_t* base; int64_t* ord; unsigned char* use; double* C; } alt_work;

static int alt_work_init(alt_work* w, int64_t n, int fc)
{
    size_t cap = (size_t)(n > 0 ? n : 1);
    w->L = (alt64*)malloc(sizeof(alt64) * cap);
    w->base = (int64_t*)malloc(sizeof(int64_t) * cap);
    w->ord = (int64_t*)malloc(sizeof(int64_t) * cap);
    w->use = (unsigned char*)malloc(cap);
    w->C = (double*)malloc(sizeof(double) * (size_t)(fc > 0 ? fc : 1));
    return w->L && w->base && w->ord && w->use && w->C;
}

static void alt_work_free(alt_work* w)
{
    free(w->L); free(w->base); free(w->ord); free(w->use); free(w->C);
}

/* The admissible outcomes of one ray (o, d): feat of[max_alts, fc], depth
 * od, opacity oo, hit count on. Returns their number, or -1 (more than
 * max_alts outcomes, a run of more than 5 ties or more than 12 optional
 * candidates) with only the definition's answer in slot 0. */
static int32_t ray_alternatives(const surfel64* s, int64_t n, const float* feats, int32_t F_total,
                                const double o[3], const double d[3], const oracle_params* P,
                                const oracle_margins* M, int32_t max_alts, alt_work* wk,
                                double* of, double* od, double* oo, int32_t* on)
{
    const int fc = P->feat_count;
    alt64* L = wk->L;
    int64_t* base = wk->base;
    int64_t* ord = wk->ord;
    unsigned char* use = wk->use;
    double* C = wk->C;
    double dn = sqrt(dot3(d, d));
    int64_t nl = 0;
    for (int64_t i = 0; i < n; ++i) {
        const surfel64* S = &s[i];
        cand64 c;
        if (S->rc2 < 0.0) continue;
        int meets = intersect(S, o, d, &c);
        if (c.den == 0.0) continue;
        int near_graze = fabs(c.den) < 2e-8 * dn;
        if (!meets && fabs(c.den) < 0.5e-8 * dn) continue;
        double rc2 = S->rc2 > 1e-12 ? S->rc2 : 1e-12;
        /* rejected whichever way a rounding goes */
        if (c.rho2 > S->rc2 + M->rho_rel * rc2) continue;
        if (c.alpha_raw < P->alpha_min - M->alpha_abs) continue;
        if (!(c.tau > P->t_min - M->t_abs) || !(c.tau < P->t_max + M->t_abs)) continue;
        double alpha = c.alpha_raw < P->alpha_max ? c.alpha_raw : P->alpha_max;
        int accepted = meets && c.rho2 <= S->rc2 && alpha >= P->alpha_min
                       && c.tau > P->t_min && c.tau < P->t_max;
        int ambiguous = !meets || near_graze || fabs(c.rho2 - S->rc2) < M->rho_rel * rc2
                        || fabs(c.alpha_raw - P->alpha_min) < M->alpha_abs
                        || fabs(c.tau - P->t_min) < M->t_abs
                        || (isfinite(P->t_max) && fabs(c.tau - P->t_max) < M->t_abs);
        if (!accepted && !ambiguous) continue;
        L[nl].tau = c.tau;
        L[nl].alpha = alpha;
        L[nl].id = i;
        L[nl].optional = ambiguous;
        L[nl].def_in = accepted;
        nl++;
    }
    qsort(L, (size_t)nl, sizeof(alt64), alt_cmp);
    for (int64_t i = 0; i < nl; ++i) base[i] = i;
    /* farthest stop: every optional candidate out, the lower threshold */
    double D, Tf;
    double Tlo = P->T_min * (1.0 - 2.0 * M->T_rel);
    int64_t far = 0;
    {
        double T = 1.0;
        int64_t i = 0;
        for (; i < nl; ++i) {
            if (L[i].optional) continue;
            T *= (1.0 - L[i].alpha);
            if (T < Tlo) break;
        }
        far = i < nl ? i : nl - 1;   /* index of the farthest possible stop hit */
    }
    int64_t kept = nl;
    if (nl > 0) {
        kept = far + 1;
        while (kept < nl) {
            double t = fabs(L[kept - 1].tau) > 1.0 ? fabs(L[kept - 1].tau) : 1.0;
            if (fabs(L[kept].tau - L[kept - 1].tau) < M->tie_abs * t) kept++;
            else break;
        }
    }
    /* optional candidates and runs of near-equal depths among the kept entries */
    int n_opt = 0;
    int opt_idx[12];
    int64_t run_start[64];
    int run_len[64];
    int n_runs = 0;
    int unresolved = 0;
    for (int64_t i = 0; i < kept; ++i) {
        if (L[i].optional) {
            if (n_opt < 12) opt_idx[n_opt] = (int)i;
            n_opt++;
        }
    }
    for (int64_t i = 0; i + 1 < kept;) {
        int64_t j = i;
        while (j + 1 < kept) {
            double t = fabs(L[j].tau) > 1.0 ? fabs(L[j].tau) : 1.0;
            if (fabs(L[j + 1].tau - L[j].tau) < M->tie_abs * t) j++;
            else break;
        }
        if (j > i) {
            if (n_runs < 64 && j - i + 1 <= 5) {
                run_start[n_runs] = i;
                run_len[n_runs] = (int)(j - i + 1);
            }
            n_runs++;
            if (j - i + 1 > 5) unresolved = 1;
        }
        i = j + 1;
    }
    double n_var = ldexp(1.0, n_opt > 12 ? 12 : n_opt);
    for (int q = 0; q < n_runs && q < 64; ++q) n_var *= factorial_d(run_len[q]);
    if (n_opt > 12 || n_runs > 64 || n_var > (double)max_alts) unresolved = 1;
    int32_t cnt = 0;
    for (int64_t v = 0; v < (unresolved ? 1 : (int64_t)n_var); ++v) {
        /* selection: bit b of v flips the definition's decision on
         * optional candidate b (v = 0 is the definition's answer) */
        for (int64_t i = 0; i < kept; ++i) use[i] = (unsigned char)L[i].def_in;
        int64_t rest = v;
        if (!unresolved) {
            for (int b = 0; b < n_opt; ++b) {
                if (rest & 1) use[opt_idx[b]] = (unsigned char)!L[opt_idx[b]].def_in;
                rest >>= 1;
            }
        }
        /* order: each run of near-equal depths permuted by its
         * Lehmer code (code 0 = the definition's (tau, id) order) */
        for (int64_t i = 0; i < kept; ++i) ord[i] = base[i];
        if (!unresolved) {
            for (int q = 0; q < n_runs; ++q) {
                int len = run_len[q];
                double f = factorial_d(len);
                int64_t code = rest % (int64_t)f;
                rest /= (int64_t)f;
                int avail[5];
                for (int a = 0; a < len; ++a) avail[a] = a;
                int left = len;
                for (int a = 0; a < len; ++a) {
                    int64_t fa = (int64_t)factorial_d(len - 1 - a);
                    int pick = (int)(code / fa);
                    code %= fa;
                    ord[run_start[q] + a] = run_start[q] + avail[pick];
                    for (int z = pick; z + 1 < left; ++z) avail[z] = avail[z + 1];
                    left--;
                }
            }
        }
        int nearT = 0;
        int64_t nc = alt_composite(L, ord, use, kept, feats, F_total, P, P->T_min, M->T_rel, C, &D, &Tf, &nearT);
        double thr[3] = {P->T_min, P->T_min * (1.0 + 2.0 * M->T_rel), P->T_min * (1.0 - 2.0 * M->T_rel)};
        int nthr = nearT ? 3 : 1;
        for (int t = 0; t < nthr; ++t) {
            if (t > 0)
                nc = alt_composite(L, ord, use, kept, feats, F_total, P, thr[t], M->T_rel, C, &D, &Tf, NULL);
            if (cnt >= max_alts) {
                unresolved = 1;
                break;
            }
            for (int c = 0; c < fc; ++c) of[(size_t)cnt * fc + c] = C[c];
            od[cnt] = D;
            oo[cnt] = 1.0 - Tf;
            on[cnt] = (int32_t)nc;
            cnt++;
        }
        if (unresolved && v > 0) break;
    }
    return unresolved ? -1 : cnt;
}

/* For R rays: the admissible outcomes (feat [R, max_alts, feat_count],
 * depth / opacity [R, max_alts], n_hits [R, max_alts]) and their number
 * count[R] (-1: more than max_alts outcomes, or a run of more than 5 ties or
 * more than 12 optional candidates; left unresolved). The first outcome is
 * always the definition's own answer. Returns 0, or -1 on bad arguments. */
int oracle_trace_alternatives(const float* means, const float* quats, const float* scales, const float* opacity,
                              const float* feats, int64_t n, int32_t F_total,
                              const float* ray_o, const float* ray_d, int64_t R,
                              const oracle_params* P, const oracle_margins* M, int32_t max_alts,
                              double* out_feat, double* out_depth, double* out_opacity, int32_t* out_nhits,
                              int32_t* out_count, int n_threads)
{
    if (n < 0 || R < 0 || !P || !M || max_alts < 1) return -1;
    if (P->feat_count > 0 && (P->feat_offset < 0 || P->feat_offset + P->feat_count > F_total)) return -1;
    surfel64* s = (surfel64*)malloc(sizeof(surfel64) * (size_t)(n > 0 ? n : 1));
    if (!s) return -1;
    load_surfels(means, quats, scales, opacity, n, P->alpha_min, s);
    nthreads_set(n_threads);
    const int fc = P->feat_count;
    int err = 0;
#pragma omp parallel
    {
        alt_work wk;
        if (!alt_work_init(&wk, n, fc)) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (int64_t r = 0; r < R; ++r) {
                double o[3] = {ray_o[3 * r], ray_o[3 * r + 1], ray_o[3 * r + 2]};
                double d[3] = {ray_d[3 * r], ray_d[3 * r + 1], ray_d[3 * r + 2]};
                out_count[r] = ray_alternatives(s, n, feats, F_total, o, d, P, M, max_alts, &wk,
                                                out_feat + (size_t)r * max_alts * (fc > 0 ? fc : 0),
                                                out_depth + (size_t)r * max_alts, out_opacity + (size_t)r * max_alts,
                                                out_nhits + (size_t)r * max_alts);
            }
        }
        alt_work_free(&wk);
    }
    free(s);
    return err ? -1 : 0;
}

/* ---------------------------------------------------------------------- */
/* Analytic gradient (the differentiable tracer of Sec. 3.3).              */
/* ---------------------------------------------------------------------- */

/* d(loss)/d(raw quaternion) from d(loss)/d(t_u, t_v, n): derivative of the
 * rotation columns with respect to (w,x,y,z), then through q/|q|. */
static void quat_backward(const surfel64* S, const double gu[3], const double gv[3], const double gn[3],
                          double gq[4])
{
    double w = S->q[0] / S->qn, x = S->q[1] / S->qn, y = S->q[2] / S->qn, z = S->q[3] / S->qn;
    /* partial derivatives of each column entry, written per component */
    double dtu_dw[3] = {0, 2 * z, -2 * y},   dtv_dw[3] = {-2 * z, 0, 2 * x},  dn_dw[3] = {2 * y, -2 * x, 0};
    double dtu_dx[3] = {0, 2 * y, 2 * z},    dtv_dx[3] = {2 * y, -4 * x, 2 * w}, dn_dx[3] = {2 * z, -2 * w, -4 * x};
    double dtu_dy[3] = {-4 * y, 2 * x, -2 * w}, dtv_dy[3] = {2 * x, 0, 2 * z}, dn_dy[3] = {2 * w, 2 * z, -4 * y};
    double dtu_dz[3] = {-4 * z, 2 * w, 2 * x}, dtv_dz[3] = {-2 * w, -4 * z, 2 * y}, dn_dz[3] = {2 * x, 2 * y, 0};
    double gh[4];
    gh[0] = dot3(gu, dtu_dw) + dot3(gv, dtv_dw) + dot3(gn, dn_dw);
    gh[1] = dot3(gu, dtu_dx) + dot3(gv, dtv_dx) + dot3(gn, dn_dx);
    gh[2] = dot3(gu, dtu_dy) + dot3(gv, dtv_dy) + dot3(gn, dn_dy);
    gh[3] = dot3(gu, dtu_dz) + dot3(gv, dtv_dz) + dot3(gn, dn_dz);
    double qh[4] = {w, x, y, z};
    double proj = qh[0] * gh[0] + qh[1] * gh[1] + qh[2] * gh[2] + qh[3] * gh[3];
    for (int k = 0; k < 4; ++k) gq[k] = (gh[k] - qh[k] * proj) / S->qn;
}

/* Backward of one ray's blend (hits[0..nc), transmittance before each hit
 * in Tl, final transmittance Tfin) for upstream gradients gC (feat_count
 * channels), gD (depth), gO (opacity); adds into the surfel gradients. The
 * suffix S_j = sum over later hits of T_m alpha_m v_m is accumulated by a
 * reverse loop over the hit list. */
static void ray_backward(const surfel64* s, const hit64* hits, int64_t nc, const double* Tl, double Tfin,
                         const float* feats, int32_t F_total, const oracle_params* P, const double o[3],
                         const double d[3], const double* gC, double gD, double gO, double* g_means,
                         double* g_quats, double* g_scales, double* g_opacity, double* g_feats)
{
    const int FC = P->feat_count;
    double S = 0.0;
    for (int64_t j = nc - 1; j >= 0; --j) {
        const surfel64* Sf = &s[hits[j].id];
        cand64 c;
        intersect(Sf, o, d, &c);
        const float* f = feats + hits[j].id * (int64_t)F_total + P->feat_offset;
        double a = hits[j].alpha, T = Tl[j];
        double v = gD * c.tau;
        for (int k = 0; k < FC; ++k) v += gC[k] * (double)f[k];
        /* dL/dalpha_j: direct term, later hits through T, final opacity */
        double dA = T * v - (S - gO * Tfin) / (1.0 - a);
        S += T * a * v;
        int64_t id = hits[j].id;
        /* features and direct depth term */
        for (int k = 0; k < FC; ++k) {
            double g = T * a * gC[k];
#pragma omp atomic
            g_feats[id * F_total + P->feat_offset + k] += g;
        }
        double g_tau = T * a * gD;
        int clamped = c.alpha_raw >= P->alpha_max;
        double g_o = clamped ? 0.0 : dA * c.G;
        double g_rho2 = clamped ? 0.0 : dA * (-0.5 * a);
        double gu = g_rho2 * 2.0 * c.u, gv = g_rho2 * 2.0 * c.v;
        /* u = e.t_u/s_u, v = e.t_v/s_v, e = o + tau d - mu, tau = n.(mu-o)/(n.d) */
        double ge[3], gmu[3], gn[3], gtu[3], gtv[3];
        for (int k = 0; k < 3; ++k) ge[k] = gu * Sf->tu[k] / Sf->su + gv * Sf->tv[k] / Sf->sv;
        double gtau_tot = g_tau + dot3(ge, d);
        for (int k = 0; k < 3; ++k) {
            gmu[k] = -ge[k] + gtau_tot * Sf->n[k] / c.den;
            gn[k] = -gtau_tot * c.e[k] / c.den;
            gtu[k] = gu * c.e[k] / Sf->su;
            gtv[k] = gv * c.e[k] / Sf->sv;
        }
        double gsu = -gu * c.u / Sf->su, gsv = -gv * c.v / Sf->sv;
        double gq[4];
        quat_backward(Sf, gtu, gtv, gn, gq);
        for (int k = 0; k < 3; ++k) {
#pragma omp atomic
            g_means[id * 3 + k] += gmu[k];
        }
        for (int k = 0; k < 4; ++k) {
#pragma omp atomic
            g_quats[id * 4 + k] += gq[k];
        }
#pragma omp atomic
        g_scales[id * 2] += gsu;
#pragma omp atomic
        g_scales[id * 2 + 1] += gsv;
#pragma omp atomic
        g_opacity[id] += g_o;
    }
}

/* Gradient of L = sum_r g_feat[r].feat[r] + g_depth[r] depth[r] + g_opac[r] opacity[r]
 * with respect to means [N,3], quats [N,4], scales [N,2], opacity [N] and
 * features [N,F_total] (only the blended channels are non-zero). FP64
 * outputs, overwritten (not accumulated). */
int oracle_trace_grad(const float* means, const float* quats, const float* scales, const float* opacity,
                      const float* feats, int64_t n, int32_t F_total,
                      const float* ray_o, const float* ray_d, int64_t R,
                      const oracle_params* P,
                      const float* g_feat, const float* g_depth, const float* g_opac,
                      double* g_means, double* g_quats, double* g_scales, double* g_opacity,
                      double* g_feats, int n_threads)
{
    if (n < 0 || R < 0 || !P || P->feat_count > 64) return -1;
    if (P->feat_count > 0 && (P->feat_offset < 0 || P->feat_offset + P->feat_count > F_total)) return -1;
    surfel64* s = (surfel64*)malloc(sizeof(surfel64) * (size_t)(n > 0 ? n : 1));
    if (!s) return -1;
    load_surfels(means, quats, scales, opacity, n, P->alpha_min, s);
    memset(g_means, 0, sizeof(double) * 3 * (size_t)n);
    memset(g_quats, 0, sizeof(double) * 4 * (size_t)n);
    memset(g_scales, 0, sizeof(double) * 2 * (size_t)n);
    memset(g_opacity, 0, sizeof(double) * (size_t)n);
    memset(g_feats, 0, sizeof(double) * (size_t)F_total * (size_t)n);
    nthreads_set(n_threads);
    const int FC = P->feat_count;
    int err = 0;
#pragma omp parallel
    {
        hit64* hits = (hit64*)malloc(sizeof(hit64) * (size_t)(n > 0 ? n : 1));
        double* Tl = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        double* C = (double*)malloc(sizeof(double) * (size_t)(FC > 0 ? FC : 1));
        if (!hits || !Tl || !C) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t r = 0; r < R; ++r) {
                double o[3] = {ray_o[3 * r], ray_o[3 * r + 1], ray_o[3 * r + 2]};
                double d[3] = {ray_d[3 * r], ray_d[3 * r + 1], ray_d[3 * r + 2]};
                int64_t nh = collect_hits(s, n, o, d, P, NULL, hits, NULL, NULL);
                double D, Tfin;
                int64_t nc = composite(hits, nh, feats, F_total, P, C, &D, &Tfin, Tl);
                double gC[64];
                for (int k = 0; k < FC; ++k) gC[k] = (double)g_feat[r * FC + k];
                ray_backward(s, hits, nc, Tl, Tfin, feats, F_total, P, o, d, gC, g_depth[r], g_opac[r],
                             g_means, g_quats, g_scales, g_opacity, g_feats);
            }
        }
        free(hits); free(Tl); free(C);
    }
    free(s);
    return err ? -1 : 0;
}

/* ---------------------------------------------------------------------- */
/* Monte Carlo rendering equation (Eq. 3, 4, 13-15).                        */
/* ---------------------------------------------------------------------- */

/* SplitMix64 stream output i (i >= 0) of `seed`: the generator advances its
 * state by the golden-ratio increment and applies the variant-13 mixer. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Uniform in [0,1) for (point p, sample s, dimension dim) with S samples per
 * point: stream index (p*S + s)*2 + dim, top 24 bits. */
static double uniform01(uint64_t seed, int64_t p, int64_t s, int64_t S, int dim)
{
    uint64_t i = ((uint64_t)p * (uint64_t)S + (uint64_t)s) * 2u + (uint64_t)dim;
    return (double)(oracle_splitmix64(seed, i) >> 40) * (1.0 / 16777216.0);
}

/* Orthonormal basis (b1, b2, n) around a unit n (Duff et al. 2017). */
static void onb(const double n[3], double b1[3], double b2[3])
{
    double sgn = n[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sgn + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sgn * n[0] * n[0] * a; b1[1] = sgn * b; b1[2] = -sgn * n[0];
    b2[0] = b; b2[1] = sgn + n[1] * n[1] * a; b2[2] = -n[1];
}

/* Cosine-weighted direction around n from (u1, u2). */
void oracle_sample_cosine(const double n[3], double u1, double u2, double out[3])
{
    double b1[3], b2[3];
    onb(n, b1, b2);
    double r = sqrt(u1), ph = 2.0 * OR_PI * u2;
    double x = r * cos(ph), y = r * sin(ph), z = sqrt(1.0 - u1 > 0.0 ? 1.0 - u1 : 0.0);
    for (int k = 0; k < 3; ++k) out[k] = x * b1[k] + y * b2[k] + z * n[k];
}

/* GGX half vector around n with alpha_g (= roughness^2) from (u1, u2). */
void oracle_sample_ggx_h(const double n[3], double alpha_g, double u1, double u2, double out[3])
{
    double b1[3], b2[3];
    onb(n, b1, b2);
    double a2 = alpha_g * alpha_g;
    double c2 = (1.0 - u1) / (1.0 + (a2 - 1.0) * u1);
    double ct = sqrt(c2), st = sqrt(1.0 - c2 > 0.0 ? 1.0 - c2 : 0.0);
    double ph = 2.0 * OR_PI * u2;
    double x = st * cos(ph), y = st * sin(ph);
    for (int k = 0; k < 3; ++k) out[k] = x * b1[k] + y * b2[k] + ct * n[k];
}

/* Equirectangular lookup, z up: phi = atan2(y,x), theta = acos(z);
 * texel coords ((phi+pi)/2pi W - 0.5, theta/pi H - 0.5); bilinear with
 * wrap in phi and clamp in theta. env is [H, W, 3]. */
/* Texels and bilinear weights of the equirectangular lookup of direction w. */
static void env_texels(int32_t H, int32_t W, const double w[3], int64_t idx[4], double wt[4])
{
    double len = sqrt(dot3(w, w));
    double z = w[2] / len;
    if (z > 1.0) z = 1.0;
    if (z < -1.0) z = -1.0;
    double phi = atan2(w[1], w[0]);
    double theta = acos(z);
    double x = (phi + OR_PI) / (2.0 * OR_PI) * W - 0.5;
    double y = theta / OR_PI * H - 0.5;
    double x0f = floor(x), y0f = floor(y);
    double fx = x - x0f, fy = y - y0f;
    int64_t x0 = (int64_t)x0f, y0 = (int64_t)y0f;
    int64_t x1 = x0 + 1, y1 = y0 + 1;
    x0 = ((x0 % W) + W) % W;
    x1 = ((x1 % W) + W) % W;
    if (y0 < 0) y0 = 0;
    if (y0 > H - 1) y0 = H - 1;
    if (y1 < 0) y1 = 0;
    if (y1 > H - 1) y1 = H - 1;
    idx[0] = y0 * W + x0; wt[0] = (1 - fy) * (1 - fx);
    idx[1] = y0 * W + x1; wt[1] = (1 - fy) * fx;
    idx[2] = y1 * W + x0; wt[2] = fy * (1 - fx);
    idx[3] = y1 * W + x1; wt[3] = fy * fx;
}

void oracle_env_lookup(const float* env, int32_t H, int32_t W, const double w[3], double out[3])
{
    int64_t idx[4];
    double wt[4];
    env_texels(H, W, w, idx, wt);
    for (int c = 0; c < 3; ++c) {
        out[c] = 0.0;
        for (int t = 0; t < 4; ++t) out[c] += wt[t] * env[idx[t] * 3 + c];
    }
}

static void normalize3(double v[3])
{
    double l = sqrt(dot3(v, v));
    v[0] /= l; v[1] /= l; v[2] /= l;
}

/* Sampling modes of the rendering-equation estimate. */
enum { MODE_SPLIT = 0, MODE_UNIFORM = 1 };

/* Incident direction of sample s of point p. MODE_SPLIT: samples below
 * n_diffuse are cosine-weighted, the rest GGX (half vector in h); returns 0
 * for a GGX sample that leaves below the horizon (no contribution, still
 * counted). MODE_UNIFORM: stratified uniform hemisphere (Eq. 15), stratum s
 * of S in cos(theta); returns 0 for a direction on the horizon. */
static int sample_direction(uint64_t seed, int64_t p, int64_t s, int64_t S, int32_t n_diffuse, int mode,
                            const double n[3], const double wo[3], double rough,
                            double wi[3], double h[3])
{
    double u1 = uniform01(seed, p, s, S, 0), u2 = uniform01(seed, p, s, S, 1);
    if (mode == MODE_UNIFORM) {
        double b1[3], b2[3];
        onb(n, b1, b2);
        double z = ((double)s + u1) / (double)S;
        double rr = sqrt(1.0 - z * z > 0.0 ? 1.0 - z * z : 0.0), ph = 2.0 * OR_PI * u2;
        for (int k = 0; k < 3; ++k) wi[k] = rr * cos(ph) * b1[k] + rr * sin(ph) * b2[k] + z * n[k];
        normalize3(wi);
        for (int k = 0; k < 3; ++k) h[k] = wi[k] + wo[k];
        normalize3(h);
        return z > 0.0;
    }
    if (s < n_diffuse) {
        oracle_sample_cosine(n, u1, u2, wi);
        normalize3(wi);
        return 1;
    }
    oracle_sample_ggx_h(n, rough * rough, u1, u2, h);
    normalize3(h);
    double oh = dot3(wo, h);
    for (int k = 0; k < 3; ++k) wi[k] = 2.0 * oh * h[k] - wo[k];
    normalize3(wi);
    if (oh <= 0.0 || dot3(wi, n) <= 0.0) return 0;
    return 1;
}

/* Directions only (for sampler tests): [P, S, 3] incident directions and a
 * validity mask [P, S]. */
int oracle_sample_dirs(const float* nrm, const float* wo_in, const float* rough, int64_t P,
                       int32_t n_diffuse, int32_t n_spec, int32_t mode, uint64_t seed, double* out_dirs,
                       int32_t* out_valid)
{
    int64_t S = (int64_t)n_diffuse + n_spec;
    for (int64_t p = 0; p < P; ++p) {
        double n[3] = {nrm[3 * p], nrm[3 * p + 1], nrm[3 * p + 2]};
        double wo[3] = {wo_in[3 * p], wo_in[3 * p + 1], wo_in[3 * p + 2]};
        normalize3(n); normalize3(wo);
        if (dot3(n, wo) <= 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
        for (int64_t s = 0; s < S; ++s) {
            double wi[3], h[3];
            int ok = sample_direction(seed, p, s, S, n_diffuse, mode, n, wo, rough[p], wi, h);
            for (int k = 0; k < 3; ++k) out_dirs[(p * S + s) * 3 + k] = wi[k];
            out_valid[p * S + s] = ok;
        }
    }
    return 0;
}

/* Specular lobe pieces at one direction (Eq. 4 with the readings above):
 * F (Schlick, on w_o.h), the two Schlick-GGX G1 factors, D (GGX) and the
 * logarithmic derivative d ln(D G) / d roughness. */
typedef struct { double F, G1i, G1o, D, dlnf_dr; } spec_terms;

static spec_terms spec_eval(double r, double ni, double no, double nh, double oh)
{
    const double F0 = 0.04;
    spec_terms t;
    double ag = r * r, a2 = ag * ag, kk = 0.5 * ag;
    double q = nh * nh * (a2 - 1.0) + 1.0;
    t.F = F0 + (1.0 - F0) * pow(1.0 - oh, 5.0);
    t.G1i = ni / (ni * (1.0 - kk) + kk);
    t.G1o = no / (no * (1.0 - kk) + kk);
    t.D = a2 / (OR_PI * q * q);
    double dlnD = 4.0 / r - 8.0 * r * r * r * nh * nh / q;
    double dlnGi = -r * (1.0 - ni) / (ni * (1.0 - kk) + kk);
    double dlnGo = -r * (1.0 - no) / (no * (1.0 - kk) + kk);
    t.dlnf_dr = dlnD + dlnGi + dlnGo;
    return t;
}

/* Upstream gradients and outputs of the surfel/env gradient of shading. */
typedef struct {
    const float* g_rgb;     /* [P,3] */
    double* g_albedo;       /* [P,3] */
    double* g_rough;        /* [P]   */
    double* g_env;          /* [H,W,3] or NULL */
    double *g_means, *g_quats, *g_scales, *g_opacity, *g_feats;
} shade_grads;

/* Monte Carlo estimate of Eq. 15 at one point, and optionally its gradient.
 * MODE_SPLIT (split-lobe importance sampling):
 *   diffuse lobe, cosine samples: f_d L_i cos / pdf = a L_i;
 *   specular lobe, GGX samples:   f_s L_i cos / pdf = F G (w_o.h) L_i / ((n.w_o)(n.h));
 * MODE_UNIFORM (Eq. 15): 2 pi / N sum (f_d + f_s) L_i (w_i.n).
 * L_i = V L_dir + L_ind with (L_ind, 1 - V) = Trace(x, w_i) (Eq. 13-14).
 * The gradient keeps the sample directions fixed: d/dr goes through f_s
 * only (d ln(D G)/dr), and each traced ray receives dL/dL_ind = g and
 * dL/dO = -g.L_dir. */
/* The per-channel factor w_c multiplying L_i of sample sI in the estimate
 * (Eq. 15 with the split or uniform estimator), and its derivatives by the
 * albedo and the roughness. Returns 1 for the samples whose traces are
 * averaged into vis / ind (the cosine samples, or all in uniform mode). */
static int sample_weight64(int mode, int64_t sI, int32_t n_diffuse, int32_t n_spec, int64_t S, const double nn[3],
                           const double wo[3], double no, const double a[3], double r, const double wi[3],
                           const double h[3], double wc[3], double dwc_da[3], double dwc_dr[3])
{
    for (int k = 0; k < 3; ++k) { dwc_da[k] = 0.0; dwc_dr[k] = 0.0; }
    if (mode == MODE_UNIFORM) {
        double ni = dot3(nn, wi), nh_ = dot3(nn, h), oh = dot3(wo, h);
        spec_terms t = spec_eval(r, ni, no, nh_, oh);
        double fs_cos = t.D * t.F * t.G1i * t.G1o / (4.0 * no);     /* f_s (w_i.n) */
        for (int k = 0; k < 3; ++k) {
            wc[k] = (2.0 * a[k] * ni + 2.0 * OR_PI * fs_cos) / (double)S;
            dwc_da[k] = 2.0 * ni / (double)S;
            dwc_dr[k] = 2.0 * OR_PI * fs_cos * t.dlnf_dr / (double)S;
        }
        return 1;
    }
    if (sI < n_diffuse) {
        for (int k = 0; k < 3; ++k) { wc[k] = a[k] / n_diffuse; dwc_da[k] = 1.0 / n_diffuse; }
        return 1;
    }
    double oh = dot3(wo, h), nh_ = dot3(nn, h), ni = dot3(nn, wi);
    spec_terms t = spec_eval(r, ni, no, nh_, oh);
    double w = t.F * t.G1i * t.G1o * oh / (no * nh_);
    for (int k = 0; k < 3; ++k) { wc[k] = w / n_spec; dwc_dr[k] = w / n_spec * t.dlnf_dr; }
    return 0;
}

static void shade_point(const surfel64* s, int64_t n, const float* feats, int32_t F_total,
                        const oracle_params* P, const oracle_margins* M, hit64* hits, near64* nears, double* Tl,
                        const double x[3], const double n_raw[3], const double wo_raw[3], const double a[3],
                        double r, int64_t key, uint64_t seed, int32_t n_diffuse, int32_t n_spec, int mode,
                        const float* env, int32_t H, int32_t W, double rgb[3], double* vis, double ind[3],
                        uint32_t* flags, const shade_grads* G, int64_t p)
{
    double nn[3] = {n_raw[0], n_raw[1], n_raw[2]}, wo[3] = {wo_raw[0], wo_raw[1], wo_raw[2]};
    normalize3(nn); normalize3(wo);
    if (dot3(nn, wo) <= 0.0) { nn[0] = -nn[0]; nn[1] = -nn[1]; nn[2] = -nn[2]; }
    const int64_t S = (int64_t)n_diffuse + n_spec;
    double no = dot3(nn, wo);
    double acc[3] = {0, 0, 0}, sum_v = 0.0, sum_i[3] = {0, 0, 0};
    double ga[3] = {0, 0, 0}, gr = 0.0;
    int64_t n_aux = 0;
    uint32_t fl = 0;
    double grgb[3] = {0, 0, 0};
    if (G) for (int k = 0; k < 3; ++k) grgb[k] = G->g_rgb[3 * p + k];
    for (int64_t sI = 0; sI < S; ++sI) {
        double wi[3], h[3];
        if (!sample_direction(seed, key, sI, S, n_diffuse, mode, nn, wo, r, wi, h)) continue;
        int64_t nnr = 0;
        int64_t nh = collect_hits(s, n, x, wi, P, M, hits, nears, &nnr);
        double C[3], D, Tfin;
        int64_t nc = composite(hits, nh, feats, F_total, P, C, &D, &Tfin, Tl);
        if (M) fl |= resolve_flags(hits, nh, nc, nears, nnr, P, M, Tl, Tfin);
        double V = Tfin;                       /* 1 - V = traced opacity */
        double Ld[3];
        oracle_env_lookup(env, H, W, wi, Ld);
        double Li[3] = {V * Ld[0] + C[0], V * Ld[1] + C[1], V * Ld[2] + C[2]};
        double wc[3], dwc_dr[3], dwc_da[3];
        int aux = sample_weight64(mode, sI, n_diffuse, n_spec, S, nn, wo, no, a, r, wi, h, wc, dwc_da, dwc_dr);
        for (int k = 0; k < 3; ++k) acc[k] += wc[k] * Li[k];
        if (aux) {
            for (int k = 0; k < 3; ++k) sum_i[k] += C[k];
            sum_v += V;
            ++n_aux;
        }
        if (G) {
            double gL[3], gO = 0.0;
            for (int k = 0; k < 3; ++k) {
                gL[k] = grgb[k] * wc[k];
                ga[k] += grgb[k] * dwc_da[k] * Li[k];
                gr += grgb[k] * dwc_dr[k] * Li[k];
                gO -= gL[k] * Ld[k];
            }
            if (G->g_env) {
                int64_t idx[4];
                double wt[4];
                env_texels(H, W, wi, idx, wt);
                for (int t4 = 0; t4 < 4; ++t4)
                    for (int k = 0; k < 3; ++k) {
#pragma omp atomic
                        G->g_env[idx[t4] * 3 + k] += wt[t4] * gL[k] * V;
                    }
            }
            ray_backward(s, hits, nc, Tl, Tfin, feats, F_total, P, x, wi, gL, 0.0, gO, G->g_means, G->g_quats,
                         G->g_scales, G->g_opacity, G->g_feats);
        }
    }
    for (int k = 0; k < 3; ++k) {
        rgb[k] = acc[k];
        ind[k] = n_aux > 0 ? sum_i[k] / (double)n_aux : 0.0;
    }
    *vis = n_aux > 0 ? sum_v / (double)n_aux : 0.0;
    *flags = fl;
    if (G) {
        for (int k = 0; k < 3; ++k) G->g_albedo[3 * p + k] = ga[k];
        G->g_rough[p] = gr;
    }
}

static int shade_args_ok(int64_t n, int64_t Pn, const oracle_params* P, int32_t F_total, int32_t n_diffuse,
                         int32_t n_spec, int32_t mode)
{
    if (n < 0 || Pn < 0 || !P || P->feat_count != 3) return 0;
    if (P->feat_offset < 0 || P->feat_offset + 3 > F_total) return 0;
    if (n_diffuse < 0 || n_spec < 0 || n_diffuse + n_spec <= 0) return 0;
    if (mode != MODE_SPLIT && mode != MODE_UNIFORM) return 0;
    if (mode == MODE_UNIFORM && n_spec != 0) return 0;
    return 1;
}

/* Monte Carlo rendering equation per G-buffer point (see shade_point).
 * Outputs rgb [P,3]; vis [P] and ind [P,3] are the means of V and L_ind
 * over the cosine samples (split mode) or over all samples (uniform mode),
 * NULL to skip; flags [P] ORs the traced rays' flags. point_ids [P] (or NULL
 * for 0..P-1) is the point number that keys the random stream of a point. */
int oracle_shade(const float* means, const float* quats, const float* scales, const float* opacity,
                 const float* feats, int64_t n, int32_t F_total,
                 const float* x_in, const float* n_in, const float* albedo, const float* rough,
                 const float* wo_in, int64_t Pn, const float* env, int32_t env_h, int32_t env_w,
                 int32_t n_diffuse, int32_t n_spec, int32_t mode, uint64_t seed, const int64_t* point_ids,
                 const oracle_params* P, const oracle_margins* M, double* out_rgb, double* out_vis,
                 double* out_ind, uint32_t* out_flags, int n_threads)
{
    if (!shade_args_ok(n, Pn, P, F_total, n_diffuse, n_spec, mode)) return -1;
    surfel64* s = (surfel64*)malloc(sizeof(surfel64) * (size_t)(n > 0 ? n : 1));
    if (!s) return -1;
    load_surfels(means, quats, scales, opacity, n, P->alpha_min, s);
    nthreads_set(n_threads);
    int err = 0;
#pragma omp parallel
    {
        hit64* hits = (hit64*)malloc(sizeof(hit64) * (size_t)(n > 0 ? n : 1));
        near64* nears = (near64*)malloc(sizeof(near64) * (size_t)(n > 0 ? n : 1));
        double* Tl = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        if (!hits || !nears || !Tl) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t p = 0; p < Pn; ++p) {
                double x[3] = {x_in[3 * p], x_in[3 * p + 1], x_in[3 * p + 2]};
                double nr[3] = {n_in[3 * p], n_in[3 * p + 1], n_in[3 * p + 2]};
                double wo[3] = {wo_in[3 * p], wo_in[3 * p + 1], wo_in[3 * p + 2]};
                double a[3] = {albedo[3 * p], albedo[3 * p + 1], albedo[3 * p + 2]};
                double rgb[3], vis, ind[3];
                uint32_t fl;
                shade_point(s, n, feats, F_total, P, M, hits, nears, Tl, x, nr, wo, a, rough[p],
                            point_ids ? point_ids[p] : p, seed, n_diffuse, n_spec, mode, env, env_h, env_w, rgb,
                            &vis, ind, &fl, NULL, p);
                for (int k = 0; k < 3; ++k) {
                    out_rgb[3 * p + k] = rgb[k];
                    if (out_ind) out_ind[3 * p + k] = ind[k];
                }
                if (out_vis) out_vis[p] = vis;
                if (out_flags) out_flags[p] = fl;
            }
        }
        free(hits); free(nears); free(Tl);
    }
    free(s);
    return err ? -1 : 0;
}

/* Admissible range of each point's estimate: every traced sample is one of
 * its ray's admissible outcomes (ray_alternatives), and the estimate is the
 * sum of the samples' terms w_c L_i (sample_weight64), so each channel lies
 * between the sums of the per-sample minima and maxima over the outcomes.
 * Outputs rgb_lo, rgb_hi [P, 3] (equal for a point with no ambiguous ray)
 * and unresolved [P] (samples whose outcomes could not all be listed; only
 * the definition's term enters for them). Returns 0, or -1 on bad
 * arguments. */
int oracle_shade_bounds(const float* means, const float* quats, const float* scales, const float* opacity,
                        const float* feats, int64_t n, int32_t F_total,
                        const float* x_in, const float* n_in, const float* albedo, const float* rough,
                        const float* wo_in, int64_t Pn, const float* env, int32_t env_h, int32_t env_w,
                        int32_t n_diffuse, int32_t n_spec, int32_t mode, uint64_t seed, const int64_t* point_ids,
                        const oracle_params* P, const oracle_margins* M, int32_t max_alts, double* rgb_lo,
                        double* rgb_hi, int32_t* unresolved, int n_threads)
{
    if (!shade_args_ok(n, Pn, P, F_total, n_diffuse, n_spec, mode) || !M || max_alts < 1) return -1;
    surfel64* s = (surfel64*)malloc(sizeof(surfel64) * (size_t)(n > 0 ? n : 1));
    if (!s) return -1;
    load_surfels(means, quats, scales, opacity, n, P->alpha_min, s);
    nthreads_set(n_threads);
    int err = 0;
#pragma omp parallel
    {
        alt_work wk;
        double* of = (double*)malloc(sizeof(double) * 3 * (size_t)max_alts);
        double* od = (double*)malloc(sizeof(double) * (size_t)max_alts);
        double* oo = (double*)malloc(sizeof(double) * (size_t)max_alts);
        int32_t* on = (int32_t*)malloc(sizeof(int32_t) * (size_t)max_alts);
        if (!alt_work_init(&wk, n, 3) || !of || !od || !oo || !on) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t p = 0; p < Pn; ++p) {
                double x[3] = {x_in[3 * p], x_in[3 * p + 1], x_in[3 * p + 2]};
                double nn[3] = {n_in[3 * p], n_in[3 * p + 1], n_in[3 * p + 2]};
                double wo[3] = {wo_in[3 * p], wo_in[3 * p + 1], wo_in[3 * p + 2]};
                double a[3] = {albedo[3 * p], albedo[3 * p + 1], albedo[3 * p + 2]};
                double r = rough[p];
                int64_t key = point_ids ? point_ids[p] : p;
                normalize3(nn);
                normalize3(wo);
                if (dot3(nn, wo) <= 0.0) { nn[0] = -nn[0]; nn[1] = -nn[1]; nn[2] = -nn[2]; }
                const int64_t S = (int64_t)n_diffuse + n_spec;
                double no = dot3(nn, wo);
                double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
                int32_t unres = 0;
                for (int64_t sI = 0; sI < S; ++sI) {
                    double wi[3], h[3];
                    if (!sample_direction(seed, key, sI, S, n_diffuse, mode, nn, wo, r, wi, h)) continue;
                    int32_t cnt = ray_alternatives(s, n, feats, F_total, x, wi, P, M, max_alts, &wk, of, od, oo, on);
                    if (cnt < 0) {
                        unres++;
                        cnt = 1;
                    }
                    double Ld[3], wc[3], dwa[3], dwr[3];
                    oracle_env_lookup(env, env_h, env_w, wi, Ld);
                    sample_weight64(mode, sI, n_diffuse, n_spec, S, nn, wo, no, a, r, wi, h, wc, dwa, dwr);
                    for (int k = 0; k < 3; ++k) {
                        double mn = INFINITY, mx = -INFINITY;
                        for (int32_t j = 0; j < cnt; ++j) {
                            double V = 1.0 - oo[j];
                            double term = wc[k] * (V * Ld[k] + of[3 * j + k]);
                            mn = term < mn ? term : mn;
                            mx = term > mx ? term : mx;
                        }
                        lo[k] += mn;
                        hi[k] += mx;
                    }
                }
                for (int k = 0; k < 3; ++k) {
                    rgb_lo[3 * p + k] = lo[k];
                    rgb_hi[3 * p + k] = hi[k];
                }
                if (unresolved) unresolved[p] = unres;
            }
        }
        alt_work_free(&wk);
        free(of); free(od); free(oo); free(on);
    }
    free(s);
    return err ? -1 : 0;
}

/* Gradient of L = sum_p g_rgb[p].rgb[p] with the sample directions fixed:
 * outputs (overwritten) g_albedo [P,3], g_rough [P], g_env [H,W,3] (or
 * NULL), and the surfel gradients through the traced rays: g_means [N,3],
 * g_quats [N,4], g_scales [N,2], g_opacity [N], g_feats [N,F] (radiance
 * channels only). */
int oracle_shade_grad(const float* means, const float* quats, const float* scales, const float* opacity,
                      const float* feats, int64_t n, int32_t F_total,
                      const float* x_in, const float* n_in, const float* albedo, const float* rough,
                      const float* wo_in, int64_t Pn, const float* env, int32_t env_h, int32_t env_w,
                      int32_t n_diffuse, int32_t n_spec, int32_t mode, uint64_t seed, const int64_t* point_ids,
                      const oracle_params* P, const float* g_rgb, double* g_albedo, double* g_rough,
                      double* g_env, double* g_means, double* g_quats, double* g_scales, double* g_opacity,
                      double* g_feats, int n_threads)
{
    if (!shade_args_ok(n, Pn, P, F_total, n_diffuse, n_spec, mode)) return -1;
    surfel64* s = (surfel64*)malloc(sizeof(surfel64) * (size_t)(n > 0 ? n : 1));
    if (!s) return -1;
    load_surfels(means, quats, scales, opacity, n, P->alpha_min, s);
    memset(g_means, 0, sizeof(double) * 3 * (size_t)n);
    memset(g_quats, 0, sizeof(double) * 4 * (size_t)n);
    memset(g_scales, 0, sizeof(double) * 2 * (size_t)n);
    memset(g_opacity, 0, sizeof(double) * (size_t)n);
    memset(g_feats, 0, sizeof(double) * (size_t)F_total * (size_t)n);
    if (g_env) memset(g_env, 0, sizeof(double) * 3 * (size_t)env_h * (size_t)env_w);
    shade_grads G = {g_rgb, g_albedo, g_rough, g_env, g_means, g_quats, g_scales, g_opacity, g_feats};
    nthreads_set(n_threads);
    int err = 0;
#pragma omp parallel
    {
        hit64* hits = (hit64*)malloc(sizeof(hit64) * (size_t)(n > 0 ? n : 1));
        near64* nears = (near64*)malloc(sizeof(near64) * (size_t)(n > 0 ? n : 1));
        double* Tl = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        if (!hits || !nears || !Tl) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t p = 0; p < Pn; ++p) {
                double x[3] = {x_in[3 * p], x_in[3 * p + 1], x_in[3 * p + 2]};
                double nr[3] = {n_in[3 * p], n_in[3 * p + 1], n_in[3 * p + 2]};
                double wo[3] = {wo_in[3 * p], wo_in[3 * p + 1], wo_in[3 * p + 2]};
                double a[3] = {albedo[3 * p], albedo[3 * p + 1], albedo[3 * p + 2]};
                double rgb[3], vis, ind[3];
                uint32_t fl;
                shade_point(s, n, feats, F_total, P, NULL, hits, nears, Tl, x, nr, wo, a, rough[p],
                            point_ids ? point_ids[p] : p, seed, n_diffuse, n_spec, mode, env, env_h, env_w, rgb,
                            &vis, ind, &fl, &G, p);
            }
        }
        free(hits); free(nears); free(Tl);
    }
    free(s);
    return err ? -1 : 0;
}

/* ====================================================================== */
/* Relighting query (supplementary "Relighting details", Eq. 18; Sec. 4,   */
/* relighting paragraph): each incident ray blends the albedo, roughness   */
/* and normal of the surfels it crosses; that aggregate surface is shaded  */
/* under the new environment with pre-integrated maps (a diffuse           */
/* irradiance map and the two split-sum factors: a roughness-prefiltered   */
/* environment and a 2D lookup table of the BRDF integral); directions are */
/* drawn by importance sampling the environment's intensity.               */
/* ====================================================================== */

/* Sizes of the pre-integrated maps. */
enum {
    RL_IRR_H = 32, RL_IRR_W = 64,             /* irradiance map                      */
    RL_LEVELS = 6,                            /* prefilter levels, roughness l / 5   */
    RL_PREF_H = 64, RL_PREF_W = 128,          /* prefiltered levels 1..5             */
    RL_LUT_N = 32,                            /* LUT cells over (n.v, roughness)     */
    RL_LUT_SAMPLES = 1024                     /* Hammersley points per LUT cell      */
};

/* Direction of the centre of texel (row, col) of an H x W equirect map. */
static void texel_dir(int64_t H, int64_t W, double row, double col, double w[3])
{
    double th = (row + 0.5) * OR_PI / (double)H;
    double ph = (col + 0.5) * 2.0 * OR_PI / (double)W - OR_PI;
    w[0] = sin(th) * cos(ph);
    w[1] = sin(th) * sin(ph);
    w[2] = cos(th);
}

/* Solid angle of any texel of row `row` (exact band area / W). */
static double texel_solid_angle(int64_t H, int64_t W, int64_t row)
{
    double t0 = row * OR_PI / (double)H, t1 = (row + 1) * OR_PI / (double)H;
    return (cos(t0) - cos(t1)) * 2.0 * OR_PI / (double)W;
}

/* Diffuse irradiance map: for each map texel centre N,
 *   Irr(N) = (1/pi) sum_t E_t max(0, w_t.N) dOmega_t
 * over all environment texels t (each of constant radiance over its solid
 * angle, seen from its centre direction w_t). out [RL_IRR_H, RL_IRR_W, 3]. */
static void relight_irradiance(const float* env, int32_t H, int32_t W, double* out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < (int64_t)RL_IRR_H * RL_IRR_W; ++i) {
        double N[3];
        texel_dir(RL_IRR_H, RL_IRR_W, (double)(i / RL_IRR_W), (double)(i % RL_IRR_W), N);
        double acc[3] = {0, 0, 0};
        for (int64_t r = 0; r < H; ++r) {
            double dO = texel_solid_angle(H, W, r);
            for (int64_t c = 0; c < W; ++c) {
                double w[3];
                texel_dir(H, W, (double)r, (double)c, w);
                double cs = dot3(w, N);
                if (cs <= 0.0) continue;
                const float* e = env + (r * W + c) * 3;
                for (int k = 0; k < 3; ++k) acc[k] += e[k] * cs * dO;
            }
        }
        for (int k = 0; k < 3; ++k) out[i * 3 + k] = acc[k] / OR_PI;
    }
}

/* GGX distribution with alpha_g = r^2 at cos(theta_h) = nh. */
static double ggx_d(double r, double nh)
{
    double a2 = r * r * r * r;
    double q = nh * nh * (a2 - 1.0) + 1.0;
    return a2 / (OR_PI * q * q);
}

/* Prefiltered environment of level l (roughness rho = l / 5, l = 1..5), the
 * radiance factor of the split sum with n = v = R: for each map texel centre R,
 *   Pref(R) = sum_t E_t D(R.h_t) max(0, w_t.R) dOmega_t
 *             / sum_t D(R.h_t) max(0, w_t.R) dOmega_t,   h_t = (w_t + R)/|w_t + R|.
 * Level 0 is the environment itself. out [RL_PREF_H, RL_PREF_W, 3]. */
static void relight_prefilter(const float* env, int32_t H, int32_t W, int level, double* out)
{
    double rho = (double)level / (double)(RL_LEVELS - 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < (int64_t)RL_PREF_H * RL_PREF_W; ++i) {
        double R[3];
        texel_dir(RL_PREF_H, RL_PREF_W, (double)(i / RL_PREF_W), (double)(i % RL_PREF_W), R);
        double acc[3] = {0, 0, 0}, wsum = 0.0;
        for (int64_t r = 0; r < H; ++r) {
            double dO = texel_solid_angle(H, W, r);
            for (int64_t c = 0; c < W; ++c) {
                double w[3];
                texel_dir(H, W, (double)r, (double)c, w);
                double cs = dot3(w, R);
                if (cs <= 0.0) continue;
                double h[3] = {w[0] + R[0], w[1] + R[1], w[2] + R[2]};
                normalize3(h);
                double wt = ggx_d(rho, dot3(R, h)) * cs * dO;
                const float* e = env + (r * W + c) * 3;
                for (int k = 0; k < 3; ++k) acc[k] += e[k] * wt;
                wsum += wt;
            }
        }
        for (int k = 0; k < 3; ++k) out[i * 3 + k] = wsum > 0.0 ? acc[k] / wsum : 0.0;
    }
}

/* Radical inverse in base 2 of i (van der Corput), for Hammersley points. */
static double radical_inverse2(uint32_t i)
{
    double r = 0.0, f = 0.5;
    while (i) {
        if (i & 1u) r += f;
        i >>= 1;
        f *= 0.5;
    }
    return r;
}

/* Split-sum BRDF table over cell centres mu = (i + 0.5)/N (= n.v) and
 * rho = (j + 0.5)/N (roughness): the BRDF-times-cosine integral
 *   int f_s (w.n) dw = F0 A(mu, rho) + B(mu, rho)
 * with Schlick F = F0 + (1 - F0)(1 - v.h)^5, split as
 *   A = int (f_s/F)(1 - (1 - v.h)^5)(w.n) dw,  B = int (f_s/F)(1 - v.h)^5 (w.n) dw,
 * estimated with RL_LUT_SAMPLES Hammersley points ((k + 0.5)/M, radical
 * inverse of k) mapped to GGX half vectors (pdf D(h) n.h), i.e. per sample
 * G (v.h)/((n.h)(n.v)) times the Fresnel part, for w = reflect(v, h) above
 * the surface. out [RL_LUT_N (mu), RL_LUT_N (rho), 2]. */
static void relight_lut(double* out)
{
    for (int i = 0; i < RL_LUT_N; ++i) {
        for (int j = 0; j < RL_LUT_N; ++j) {
            double mu = (i + 0.5) / RL_LUT_N, rho = (j + 0.5) / RL_LUT_N;
            double ag = rho * rho, a2 = ag * ag, kk = 0.5 * ag;
            double v[3] = {sqrt(1.0 - mu * mu), 0.0, mu};
            double A = 0.0, B = 0.0;
            for (int s = 0; s < RL_LUT_SAMPLES; ++s) {
                double u1 = (s + 0.5) / RL_LUT_SAMPLES, u2 = radical_inverse2((uint32_t)s);
                double c2 = (1.0 - u1) / (1.0 + (a2 - 1.0) * u1);
                double ct = sqrt(c2), st = sqrt(1.0 - c2 > 0.0 ? 1.0 - c2 : 0.0);
                double ph = 2.0 * OR_PI * u2;
                double h[3] = {st * cos(ph), st * sin(ph), ct};
                double vh = dot3(v, h);
                double l[3] = {2.0 * vh * h[0] - v[0], 2.0 * vh * h[1] - v[1], 2.0 * vh * h[2] - v[2]};
                if (l[2] <= 0.0 || vh <= 0.0) continue;
                double G = (l[2] / (l[2] * (1.0 - kk) + kk)) * (mu / (mu * (1.0 - kk) + kk));
                double gv = G * vh / (h[2] * mu);
                double fc = pow(1.0 - vh, 5.0);
                A += (1.0 - fc) * gv;
                B += fc * gv;
            }
            out[(i * RL_LUT_N + j) * 2] = A / RL_LUT_SAMPLES;
            out[(i * RL_LUT_N + j) * 2 + 1] = B / RL_LUT_SAMPLES;
        }
    }
}

/* Importance-sampling tables of the environment: texel weight
 * w_t = lum(E_t) sin(theta of the row centre), lum = 0.2126 r + 0.7152 g +
 * 0.0722 b. row_cdf[r] = sum of the weights of rows < r (H + 1 entries);
 * col_cdf[r (W+1) + c] = sum of the weights of texels (r, < c). */
static void relight_cdf(const float* env, int32_t H, int32_t W, double* row_cdf, double* col_cdf)
{
    row_cdf[0] = 0.0;
    for (int64_t r = 0; r < H; ++r) {
        double s = sin((r + 0.5) * OR_PI / (double)H);
        double* cc = col_cdf + r * (W + 1);
        cc[0] = 0.0;
        for (int64_t c = 0; c < W; ++c) {
            const float* e = env + (r * W + c) * 3;
            double lum = 0.2126 * e[0] + 0.7152 * e[1] + 0.0722 * e[2];
            cc[c + 1] = cc[c] + lum * s;
        }
        row_cdf[r + 1] = row_cdf[r] + cc[W];
    }
}

/* Largest index k in [0, n) with cdf[k] <= t and cdf[k+1] > cdf[k]
 * (cdf has n + 1 non-decreasing entries, cdf[0] <= t < cdf[n]). */
static int64_t cdf_find(const double* cdf, int64_t n, double t)
{
    int64_t lo = 0, hi = n;   /* invariant: cdf[lo] <= t < cdf[hi] */
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) / 2;
        if (cdf[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

/* Environment sample from (u1, u2): row by the row cdf at u1 total, column
 * by that row's cdf at u2 (row total); the fractions left over place the
 * direction inside the texel uniformly in (phi, theta):
 *   theta = (row + f_v) pi / H, phi = (col + f_u) 2 pi / W - pi,
 * pdf (solid angle) = (w_t / total) W H / (2 pi^2 sin theta).
 * Returns 0 if the environment has no weight. */
static int env_sample(const double* row_cdf, const double* col_cdf, int32_t H, int32_t W, double u1, double u2,
                      double w[3], double* pdf)
{
    double total = row_cdf[H];
    if (!(total > 0.0)) return 0;
    double t1 = u1 * total;
    int64_t r = cdf_find(row_cdf, H, t1);
    const double* cc = col_cdf + r * (W + 1);
    double rw = cc[W];
    double fv = (t1 - row_cdf[r]) / rw;
    double t2 = u2 * rw;
    int64_t c = cdf_find(cc, W, t2);
    double wt = cc[c + 1] - cc[c];
    double fu = (t2 - cc[c]) / wt;
    double th = (r + fv) * OR_PI / (double)H;
    double ph = (c + fu) * 2.0 * OR_PI / (double)W - OR_PI;
    double sth = sin(th);
    w[0] = sth * cos(ph);
    w[1] = sth * sin(ph);
    w[2] = cos(th);
    *pdf = sth > 0.0 ? (wt / total) * (double)W * (double)H / (2.0 * OR_PI * OR_PI * sth) : 0.0;
    return *pdf > 0.0;
}

/* Bilinear lookup of an h x w x 3 double map at direction d (same equirect
 * convention as the environment). */
static void map_lookup(const double* map, int32_t h, int32_t w, const double d[3], double out[3])
{
    int64_t idx[4];
    double wt[4];
    env_texels(h, w, d, idx, wt);
    for (int k = 0; k < 3; ++k) {
        out[k] = 0.0;
        for (int t = 0; t < 4; ++t) out[k] += wt[t] * map[idx[t] * 3 + k];
    }
}

/* Bilinear lookup of the LUT at (mu, rho), coordinates clamped to the cell
 * centres. */
static void lut_lookup(const double* lut, double mu, double rho, double* A, double* B)
{
    double x = mu * RL_LUT_N - 0.5, y = rho * RL_LUT_N - 0.5;
    if (x < 0.0) x = 0.0;
    if (x > RL_LUT_N - 1) x = RL_LUT_N - 1;
    if (y < 0.0) y = 0.0;
    if (y > RL_LUT_N - 1) y = RL_LUT_N - 1;
    int i0 = (int)floor(x), j0 = (int)floor(y);
    if (i0 > RL_LUT_N - 2) i0 = RL_LUT_N - 2;
    if (j0 > RL_LUT_N - 2) j0 = RL_LUT_N - 2;
    double fx = x - i0, fy = y - j0;
    double v[2];
    for (int k = 0; k < 2; ++k) {
        double a = lut[(i0 * RL_LUT_N + j0) * 2 + k], b = lut[(i0 * RL_LUT_N + j0 + 1) * 2 + k];
        double c = lut[((i0 + 1) * RL_LUT_N + j0) * 2 + k], d = lut[((i0 + 1) * RL_LUT_N + j0 + 1) * 2 + k];
        v[k] = (1 - fx) * ((1 - fy) * a + fy * b) + fx * ((1 - fy) * c + fy * d);
    }
    *A = v[0];
    *B = v[1];
}

/* Pre-integrated maps of one environment. */
typedef struct {
    double irr[RL_IRR_H * RL_IRR_W * 3];
    double pref[(RL_LEVELS - 1) * RL_PREF_H * RL_PREF_W * 3];
    double lut[RL_LUT_N * RL_LUT_N * 2];
} relight_maps;

/* Split-sum prefiltered radiance in direction d at roughness rho: linear
 * between the two nearest levels (level 0 = the environment, bilinear). */
static void pref_lookup(const relight_maps* M, const float* env, int32_t H, int32_t W, const double d[3],
                        double rho, double out[3])
{
    if (rho < 0.0) rho = 0.0;
    if (rho > 1.0) rho = 1.0;
    double t = rho * (RL_LEVELS - 1);
    int l0 = (int)floor(t);
    if (l0 > RL_LEVELS - 2) l0 = RL_LEVELS - 2;
    double f = t - l0;
    double a[3], b[3];
    if (l0 == 0)
        oracle_env_lookup(env, H, W, d, a);
    else
        map_lookup(M->pref + (size_t)(l0 - 1) * RL_PREF_H * RL_PREF_W * 3, RL_PREF_H, RL_PREF_W, d, a);
    map_lookup(M->pref + (size_t)l0 * RL_PREF_H * RL_PREF_W * 3, RL_PREF_H, RL_PREF_W, d, b);
    for (int k = 0; k < 3; ++k) out[k] = (1.0 - f) * a[k] + f * b[k];
}

/* Exported maps (for pins and for the GPU maps' parity): irr [32,64,3],
 * pref [5,64,128,3] (levels 1..5), lut [32,32,2], row_cdf [H+1],
 * col_cdf [H, W+1]; any pointer may be NULL. */
int oracle_relight_maps(const float* env, int32_t H, int32_t W, int n_threads, double* irr, double* pref,
                        double* lut, double* row_cdf, double* col_cdf)
{
    if (H <= 0 || W <= 0 || !env) return -1;
    nthreads_set(n_threads);
    if (irr) relight_irradiance(env, H, W, irr);
    if (pref)
        for (int l = 1; l < RL_LEVELS; ++l)
            relight_prefilter(env, H, W, l, pref + (size_t)(l - 1) * RL_PREF_H * RL_PREF_W * 3);
    if (lut) relight_lut(lut);
    if (row_cdf && col_cdf) relight_cdf(env, H, W, row_cdf, col_cdf);
    return 0;
}

/* Environment samples only (for sampler pins): dirs [P, S, 3], pdf [P, S]. */
int oracle_env_samples(const float* env, int32_t H, int32_t W, int64_t P, int32_t S, uint64_t seed,
                       double* dirs, double* pdf)
{
    double* row_cdf = (double*)malloc(sizeof(double) * (size_t)(H + 1));
    double* col_cdf = (double*)malloc(sizeof(double) * (size_t)H * (size_t)(W + 1));
    if (!row_cdf || !col_cdf) { free(row_cdf); free(col_cdf); return -1; }
    relight_cdf(env, H, W, row_cdf, col_cdf);
    for (int64_t p = 0; p < P; ++p)
        for (int64_t s = 0; s < S; ++s) {
            double w[3] = {0, 0, 1}, q = 0.0;
            env_sample(row_cdf, col_cdf, H, W, uniform01(seed, p, s, S, 0), uniform01(seed, p, s, S, 1), w, &q);
            for (int k = 0; k < 3; ++k) dirs[(p * S + s) * 3 + k] = w[k];
            pdf[p * S + s] = q;
        }
    free(row_cdf);
    free(col_cdf);
    return 0;
}

/* Relighting estimate at each point (the point's own BRDF as in the
 * shading estimate; n flipped towards w_o):
 *   rgb = 1/S sum_s f(w_s, w_o) L_i(w_s) max(0, w_s.n) / pdf(w_s),
 * w_s drawn from the environment tables with uniforms (p S + s) 2 + dim of
 * `seed`. L_i = V E(w) + L_ind with (V, and the blended material) from
 * tracing (x, w): O = 1 - V, A_r = sum(w a)/O, R_r = sum(w r)/O, N_r the
 * normalised sum(w n) (the paper's normalised blend weights), flipped to
 * face v = -w; L_ind = O (A_r Irr(N_r) + Pref(reflect(v, N_r), R_r)
 * (F0 LUT_A(N_r.v, R_r) + LUT_B(N_r.v, R_r))), F0 = 0.04. The traced
 * channels (params feat_offset, feat_count = 7) are [a (3), r, n (3)].
 * Outputs rgb [P,3]; vis [P] and ind [P,3] are means over all samples;
 * flags [P] ORs the traced rays' ambiguity flags. */
/* One relighting sample w (density pdf) whose trace gave the blended
 * material channels C[7] = [albedo (3), roughness, normal (3)] sums and the
 * transmittance V: the indirect light of the traced surface, Lind, and the
 * sample's term of the estimate, term = (a/pi + f_s) (V E + Lind) (n.w) / pdf
 * (0 below the horizon). */
static void relight_sample_term(const relight_maps* maps, const float* env, int32_t H, int32_t W,
                                const double w[3], double pdf, const double C[7], double V, const double nn[3],
                                const double wo[3], double no, const double a[3], double r, double term[3],
                                double Lind[3])
{
    double O = 1.0 - V;
    for (int k = 0; k < 3; ++k) { Lind[k] = 0.0; term[k] = 0.0; }
    if (O > 0.0) {
        double Ar[3] = {C[0] / O, C[1] / O, C[2] / O}, Rr = C[3] / O;
        double Nr[3] = {C[4], C[5], C[6]}, v[3] = {-w[0], -w[1], -w[2]};
        double len = sqrt(dot3(Nr, Nr));
        if (len > 1e-12) {
            for (int k = 0; k < 3; ++k) Nr[k] /= len;
        } else {
            for (int k = 0; k < 3; ++k) Nr[k] = v[k];
        }
        if (dot3(Nr, v) < 0.0) for (int k = 0; k < 3; ++k) Nr[k] = -Nr[k];
        double mu = dot3(Nr, v);
        if (mu > 1.0) mu = 1.0;
        double refl[3], irr[3], pref[3], LA, LB;
        for (int k = 0; k < 3; ++k) refl[k] = 2.0 * mu * Nr[k] - v[k];
        map_lookup(maps->irr, RL_IRR_H, RL_IRR_W, Nr, irr);
        pref_lookup(maps, env, H, W, refl, Rr, pref);
        lut_lookup(maps->lut, mu, Rr, &LA, &LB);
        for (int k = 0; k < 3; ++k) Lind[k] = O * (Ar[k] * irr[k] + pref[k] * (0.04 * LA + LB));
    }
    double E[3];
    oracle_env_lookup(env, H, W, w, E);
    double ni = dot3(nn, w);
    if (ni <= 0.0) return;
    double h[3] = {w[0] + wo[0], w[1] + wo[1], w[2] + wo[2]};
    normalize3(h);
    spec_terms t = spec_eval(r, ni, no, dot3(nn, h), dot3(wo, h));
    double fs = t.D * t.F * t.G1i * t.G1o / (4.0 * ni * no);
    for (int k = 0; k < 3; ++k) term[k] = (a[k] / OR_PI + fs) * (V * E[k] + Lind[k]) * ni / pdf;
}

int oracle_relight(const float* means, const float* quats, const float* scales, const float* opacity,
                   const float* feats, int64_t n, int32_t F_total,
                   const float* x_in, const float* n_in, const float* albedo, const float* rough,
                   const float* wo_in, int64_t Pn, const float* env, int32_t H, int32_t W, int32_t S,
                   uint64_t seed, const int64_t* point_ids, const oracle_params* P, const oracle_margins* M,
                   double* out_rgb, double* out_vis, double* out_ind, uint32_t* out_flags, int n_threads)
{
    if (n < 0 || Pn < 0 || !P || P->feat_count != 7 || S <= 0 || H <= 0 || W <= 0) return -1;
    if (P->feat_offset < 0 || P->feat_offset + 7 > F_total) return -1;
    relight_maps* maps = (relight_maps*)malloc(sizeof(relight_maps));
    double* row_cdf = (double*)malloc(sizeof(double) * (size_t)(H + 1));
    double* col_cdf = (double*)malloc(sizeof(double) * (size_t)H * (size_t)(W + 1));
    surfel64* s = (surfel64*)malloc(sizeof(surfel64) * (size_t)(n > 0 ? n : 1));
    if (!maps || !row_cdf || !col_cdf || !s) {
        free(maps); free(row_cdf); free(col_cdf); free(s);
        return -1;
    }
    oracle_relight_maps(env, H, W, n_threads, maps->irr, maps->pref, maps->lut, row_cdf, col_cdf);
    load_surfels(means, quats, scales, opacity, n, P->alpha_min, s);
    nthreads_set(n_threads);
    int err = 0;
#pragma omp parallel
    {
        hit64* hits = (hit64*)malloc(sizeof(hit64) * (size_t)(n > 0 ? n : 1));
        near64* nears = (near64*)malloc(sizeof(near64) * (size_t)(n > 0 ? n : 1));
        double* Tl = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        if (!hits || !nears || !Tl) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t p = 0; p < Pn; ++p) {
                double x[3] = {x_in[3 * p], x_in[3 * p + 1], x_in[3 * p + 2]};
                double nn[3] = {n_in[3 * p], n_in[3 * p + 1], n_in[3 * p + 2]};
                double wo[3] = {wo_in[3 * p], wo_in[3 * p + 1], wo_in[3 * p + 2]};
                double a[3] = {albedo[3 * p], albedo[3 * p + 1], albedo[3 * p + 2]};
                double r = rough[p];
                int64_t key = point_ids ? point_ids[p] : p;
                normalize3(nn);
                normalize3(wo);
                if (dot3(nn, wo) <= 0.0) { nn[0] = -nn[0]; nn[1] = -nn[1]; nn[2] = -nn[2]; }
                double no = dot3(nn, wo);
                double acc[3] = {0, 0, 0}, sv = 0.0, si[3] = {0, 0, 0};
                uint32_t fl = 0;
                for (int64_t sI = 0; sI < S; ++sI) {
                    double w[3], pdf;
                    if (!env_sample(row_cdf, col_cdf, H, W, uniform01(seed, key, sI, S, 0),
                                    uniform01(seed, key, sI, S, 1), w, &pdf))
                        continue;
                    int64_t nnr = 0;
                    int64_t nh = collect_hits(s, n, x, w, P, M, hits, nears, &nnr);
                    double C[7], D, Tfin;
                    int64_t nc = composite(hits, nh, feats, F_total, P, C, &D, &Tfin, Tl);
                    if (M) fl |= resolve_flags(hits, nh, nc, nears, nnr, P, M, Tl, Tfin);
                    double term[3], Lind[3];
                    relight_sample_term(maps, env, H, W, w, pdf, C, Tfin, nn, wo, no, a, r, term, Lind);
                    sv += Tfin;
                    for (int k = 0; k < 3; ++k) {
                        si[k] += Lind[k];
                        acc[k] += term[k];
                    }
                }
                for (int k = 0; k < 3; ++k) {
                    out_rgb[3 * p + k] = acc[k] / (double)S;
                    if (out_ind) out_ind[3 * p + k] = si[k] / (double)S;
                }
                if (out_vis) out_vis[p] = sv / (double)S;
                if (out_flags) out_flags[p] = fl;
            }
        }
        free(hits); free(nears); free(Tl);
    }
    free(maps); free(row_cdf); free(col_cdf); free(s);
    return err ? -1 : 0;
}

/* Admissible range of each point's relighting estimate (as
 * oracle_shade_bounds for oracle_shade): every traced sample is one of its
 * ray's admissible outcomes of the 7 material channels and the opacity, and
 * the estimate is (1/S) times the sum of the samples' terms, so each channel
 * lies between the sums of the per-sample minima and maxima. Outputs
 * rgb_lo, rgb_hi [P, 3] and unresolved [P] (samples whose outcomes could not
 * all be listed; only the definition's term enters for them). */
int oracle_relight_bounds(const float* means, const float* quats, const float* scales, const float* opacity,
                          const float* feats, int64_t n, int32_t F_total,
                          const float* x_in, const float* n_in, const float* albedo, const float* rough,
                          const float* wo_in, int64_t Pn, const float* env, int32_t H, int32_t W, int32_t S,
                          uint64_t seed, const int64_t* point_ids, const oracle_params* P, const oracle_margins* M,
                          int32_t max_alts, double* rgb_lo, double* rgb_hi, int32_t* unresolved, int n_threads)
{
    if (n < 0 || Pn < 0 || !P || !M || P->feat_count != 7 || S <= 0 || H <= 0 || W <= 0 || max_alts < 1) return -1;
    if (P->feat_offset < 0 || P->feat_offset + 7 > F_total) return -1;
    relight_maps* maps = (relight_maps*)malloc(sizeof(relight_maps));
    double* row_cdf = (double*)malloc(sizeof(double) * (size_t)(H + 1));
    double* col_cdf = (double*)malloc(sizeof(double) * (size_t)H * (size_t)(W + 1));
    surfel64* s = (surfel64*)malloc(sizeof(surfel64) * (size_t)(n > 0 ? n : 1));
    if (!maps || !row_cdf || !col_cdf || !s) {
        free(maps); free(row_cdf); free(col_cdf); free(s);
        return -1;
    }
    oracle_relight_maps(env, H, W, n_threads, maps->irr, maps->pref, maps->lut, row_cdf, col_cdf);
    load_surfels(means, quats, scales, opacity, n, P->alpha_min, s);
    nthreads_set(n_threads);
    int err = 0;
#pragma omp parallel
    {
        alt_work wk;
        double* of = (double*)malloc(sizeof(double) * 7 * (size_t)max_alts);
        double* od = (double*)malloc(sizeof(double) * (size_t)max_alts);
        double* oo = (double*)malloc(sizeof(double) * (size_t)max_alts);
        int32_t* on = (int32_t*)malloc(sizeof(int32_t) * (size_t)max_alts);
        if (!alt_work_init(&wk, n, 7) || !of || !od || !oo || !on) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t p = 0; p < Pn; ++p) {
                double x[3] = {x_in[3 * p], x_in[3 * p + 1], x_in[3 * p + 2]};
                double nn[3] = {n_in[3 * p], n_in[3 * p + 1], n_in[3 * p + 2]};
                double wo[3] = {wo_in[3 * p], wo_in[3 * p + 1], wo_in[3 * p + 2]};
                double a[3] = {albedo[3 * p], albedo[3 * p + 1], albedo[3 * p + 2]};
                double r = rough[p];
                int64_t key = point_ids ? point_ids[p] : p;
                normalize3(nn);
                normalize3(wo);
                if (dot3(nn, wo) <= 0.0) { nn[0] = -nn[0]; nn[1] = -nn[1]; nn[2] = -nn[2]; }
                double no = dot3(nn, wo);
                double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
                int32_t unres = 0;
                for (int64_t sI = 0; sI < S; ++sI) {
                    double w[3], pdf;
                    if (!env_sample(row_cdf, col_cdf, H, W, uniform01(seed, key, sI, S, 0),
                                    uniform01(seed, key, sI, S, 1), w, &pdf))
                        continue;
                    int32_t cnt = ray_alternatives(s, n, feats, F_total, x, w, P, M, max_alts, &wk, of, od, oo, on);
                    if (cnt < 0) {
                        unres++;
                        cnt = 1;
                    }
                    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
                    for (int32_t j = 0; j < cnt; ++j) {
                        double term[3], Lind[3];
                        relight_sample_term(maps, env, H, W, w, pdf, of + 7 * (size_t)j, 1.0 - oo[j], nn, wo, no, a,
                                            r, term, Lind);
                        for (int k = 0; k < 3; ++k) {
                            mn[k] = term[k] < mn[k] ? term[k] : mn[k];
                            mx[k] = term[k] > mx[k] ? term[k] : mx[k];
                        }
                    }
                    for (int k = 0; k < 3; ++k) {
                        lo[k] += mn[k];
                        hi[k] += mx[k];
                    }
                }
                for (int k = 0; k < 3; ++k) {
                    rgb_lo[3 * p + k] = lo[k] / (double)S;
                    rgb_hi[3 * p + k] = hi[k] / (double)S;
                }
                if (unresolved) unresolved[p] = unres;
            }
        }
        alt_work_free(&wk);
        free(of); free(od); free(oo); free(on);
    }
    free(maps); free(row_cdf); free(col_cdf); free(s);
    return err ? -1 : 0;
}

/* ====================================================================== */
/* 2D Gaussian rasterisation of a G-buffer (Sec. 3.3 stage I/II: the maps  */
/* of Eq. 9 are rendered by 2DGS rasterisation, which blends Eq. 2 in the  */
/* order of the splats' centre depths rather than of the per-pixel         */
/* intersection depths, with the 2DGS screen-space low-pass filter).       */
/* ====================================================================== */

/* Pinhole camera (the same convention as the CUDA library's camera rays). */
typedef struct {
    float origin[3], forward[3], right[3], up[3];
    float tan_half_fov;
    int32_t width, height;
} oracle_camera;

typedef struct { double z; int64_t id; } zkey64;

static int zkey_cmp(const void* a, const void* b)
{
    const zkey64* x = (const zkey64*)a;
    const zkey64* y = (const zkey64*)b;
    if (x->z < y->z) return -1;
    if (x->z > y->z) return 1;
    return (x->id < y->id) ? -1 : (x->id > y->id);
}

/* Extra flag of the rasteriser: the 3D and screen-space terms of rho^2 are
 * within the margin of each other (the blended depth switches between the
 * intersection and the centre there). */
enum { OF_BRANCH = 128u };

/* Rasterise: for every pixel (px, py) of a width x height image (row-major
 * output), with the camera ray d of that pixel (unit; the camera's formula in
 * FP64), the surfels whose centre has view depth z_c = (mu - o).forward >
 * t_min are blended in ascending (z_c, user index) order. Per surfel:
 *   rho3^2 = u^2 + v^2 of the ray-plane intersection (Eq. 6-7) when
 *            |n.d| >= 1e-8 and tau > 0, else +inf;
 *   rho2^2 = |(px, py) - c|^2 / sigma^2, c the projected centre in pixel
 *            coordinates (pixel centres at integers), sigma^2 = 1/2 (the
 *            2DGS low-pass filter);
 *   rho^2 = min(rho3^2, rho2^2); kept if rho^2 <= rho_c^2 and
 *   alpha = min(alpha_max, o exp(-rho^2/2)) >= alpha_min; its depth is tau
 *   if rho3^2 <= rho2^2, else (mu - o).d.
 * Blending as the tracer (w = T alpha, stop after the hit that makes
 * T < T_min). Outputs per pixel: feat [fc], depth, opacity 1 - T, n_hits,
 * flags. */
int oracle_rasterize(const float* means, const float* quats, const float* scales, const float* opacity,
                     const float* feats, int64_t n, int32_t F_total, const oracle_camera* cam,
                     const oracle_params* P, const oracle_margins* M, double* out_feat, double* out_depth,
                     double* out_opacity, int32_t* out_nhits, uint32_t* out_flags, int n_threads)
{
    if (!cam || !P || n < 0 || cam->width <= 0 || cam->height <= 0) return -1;
    if (P->feat_count < 0 || P->feat_offset < 0 || P->feat_offset + P->feat_count > F_total) return -1;
    surfel64* s = (surfel64*)malloc(sizeof(surfel64) * (size_t)(n > 0 ? n : 1));
    zkey64* order = (zkey64*)malloc(sizeof(zkey64) * (size_t)(n > 0 ? n : 1));
    if (!s || !order) { free(s); free(order); return -1; }
    load_surfels(means, quats, scales, opacity, n, P->alpha_min, s);
    double o[3], fw[3], rt[3], up[3];
    for (int k = 0; k < 3; ++k) {
        o[k] = cam->origin[k]; fw[k] = cam->forward[k]; rt[k] = cam->right[k]; up[k] = cam->up[k];
    }
    const double W = cam->width, H = cam->height, tf = cam->tan_half_fov, aspect = W / H;
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        double mo[3] = {s[i].mu[0] - o[0], s[i].mu[1] - o[1], s[i].mu[2] - o[2]};
        double z = dot3(mo, fw);
        if (!(z > P->t_min) || s[i].rc2 < 0.0) continue;
        order[m].z = z;
        order[m].id = i;
        ++m;
    }
    qsort(order, (size_t)m, sizeof(zkey64), zkey_cmp);
    const double sigma2 = 0.5;
    nthreads_set(n_threads);
    const int64_t npix = (int64_t)cam->width * cam->height;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t pix = 0; pix < npix; ++pix) {
        const int64_t py = pix / cam->width, px = pix % cam->width;
        double sx = (px + 0.5) / W * 2.0 - 1.0, sy = 1.0 - (py + 0.5) / H * 2.0;
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = fw[k] + sx * tf * aspect * rt[k] + sy * tf * up[k];
        normalize3(d);
        double T = 1.0, D = 0.0, C[64];
        for (int c = 0; c < P->feat_count; ++c) C[c] = 0.0;
        int32_t nh = 0;
        uint32_t fl = 0;
        double z_prev = -1.0;
        for (int64_t j = 0; j < m; ++j) {
            const surfel64* S = &s[order[j].id];
            double mo[3] = {S->mu[0] - o[0], S->mu[1] - o[1], S->mu[2] - o[2]};
            double zc = order[j].z;
            double pxc = (dot3(mo, rt) / zc / (tf * aspect) + 1.0) * 0.5 * W - 0.5;
            double pyc = (1.0 - dot3(mo, up) / zc / tf) * 0.5 * H - 0.5;
            double rho2d = ((px - pxc) * (px - pxc) + (py - pyc) * (py - pyc)) / sigma2;
            cand64 c;
            double rho3d = INFINITY;
            int hit3 = intersect(S, o, d, &c) && c.tau > 0.0;
            if (hit3) rho3d = c.rho2;
            double rho2 = rho3d < rho2d ? rho3d : rho2d;
            double araw = S->o * exp(-0.5 * rho2);
            if (M) {
                uint32_t kind = 0;
                if (fabs(rho2 - S->rc2) < M->rho_rel * (S->rc2 > 1e-12 ? S->rc2 : 1e-12)) kind |= OF_RHO;
                if (fabs(araw - P->alpha_min) < M->alpha_abs) kind |= OF_ALPHA;
                if (fabs(araw - P->alpha_max) < M->clamp_abs) kind |= OF_CLAMP;
                if (hit3 && fabs(rho3d - rho2d) < M->rho_rel * (rho2 > 1e-12 ? rho2 : 1e-12)) kind |= OF_BRANCH;
                if (fabs(c.den) < 2e-8 && fabs(c.den) >= 0.5e-8) kind |= OF_GRAZE;
                if (hit3 && fabs(c.tau) < M->t_abs) kind |= OF_TRANGE;
                fl |= kind;
            }
            if (rho2 > S->rc2) continue;
            double alpha = araw < P->alpha_max ? araw : P->alpha_max;
            if (alpha < P->alpha_min) continue;
            if (M && z_prev >= 0.0 && fabs(zc - z_prev) < M->tie_abs * (zc > 1.0 ? zc : 1.0)) fl |= OF_TIE;
            z_prev = zc;
            double depth = rho3d <= rho2d ? c.tau : dot3(mo, d);
            double w = T * alpha;
            const float* f = feats + order[j].id * (int64_t)F_total + P->feat_offset;
            for (int cc = 0; cc < P->feat_count; ++cc) C[cc] += w * (double)f[cc];
            D += w * depth;
            double Tn = T * (1.0 - alpha);
            if (M && fabs(Tn - P->T_min) < M->T_rel * P->T_min) fl |= OF_T;
            T = Tn;
            ++nh;
            if (T < P->T_min) break;
        }
        for (int cc = 0; cc < P->feat_count; ++cc) out_feat[pix * P->feat_count + cc] = C[cc];
        out_depth[pix] = D;
        out_opacity[pix] = 1.0 - T;
        out_nhits[pix] = nh;
        if (out_flags) out_flags[pix] = fl;
    }
    free(s);
    free(order);
    return 0;
}
