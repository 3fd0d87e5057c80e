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
        /* per-channel factor w_c multiplying L_i in the estimate, and d w_c / d r */
        double wc[3], dwc_dr[3] = {0, 0, 0}, dwc_da[3] = {0, 0, 0};
        int aux = 0;
        if (mode == MODE_UNIFORM) {
            double ni = dot3(nn, wi), nh_ = dot3(nn, h), oh = dot3(wo, h);
            spec_terms t = spec_eval(r, ni, no, nh_, oh);
            double fs_cos = t.D * t.F * t.G1i * t.G1o / (4.0 * no);     /* f_s (w_i.n) */
            for (int k = 0; k < 3; ++k) {
                wc[k] = (2.0 * a[k] * ni + 2.0 * OR_PI * fs_cos) / (double)S;
                dwc_da[k] = 2.0 * ni / (double)S;
                dwc_dr[k] = 2.0 * OR_PI * fs_cos * t.dlnf_dr / (double)S;
            }
            aux = 1;
        } else if (sI < n_diffuse) {
            for (int k = 0; k < 3; ++k) { wc[k] = a[k] / n_diffuse; dwc_da[k] = 1.0 / n_diffuse; }
            aux = 1;
        } else {
            double oh = dot3(wo, h), nh_ = dot3(nn, h), ni = dot3(nn, wi);
            spec_terms t = spec_eval(r, ni, no, nh_, oh);
            double w = t.F * t.G1i * t.G1o * oh / (no * nh_);
            for (int k = 0; k < 3; ++k) { wc[k] = w / n_spec; dwc_dr[k] = w / n_spec * t.dlnf_dr; }
        }
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
