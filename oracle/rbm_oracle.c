/*
 * Plain FP64 CPU oracle of the Random Batch Method RBM-1 and of the direct
 * O(N^2) forward-Euler step (Jin, Li & Liu, "Random Batch Methods (RBM) for
 * interacting particle systems", arXiv:1812.10575).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link
 * or call this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no source with the CUDA library.
 *
 * Every routine is written for a reader checking it against the paper by eye:
 * plain loops, no blocking, no fusion.  Sums over particles run in ascending
 * particle-id order so that RBM with p = N reproduces the direct step bit for
 * bit.  Particle loops may run on several OpenMP threads; every particle's
 * result is computed by one thread from read-only inputs, so the output does
 * not depend on the thread count.
 *
 * Conventions (the readings of the paper this oracle fixes):
 *   - model (Sec. 1, eq. "interactingps"):
 *       dX^i = -grad V(X^i) dt + 1/(N-1) sum_{j != i} K(X^i - X^j) dt + sigma dB^i
 *   - RBM-1 (Sec. 2.1, Algorithm "randomdiv", eq. "firstalgorithm"): per step,
 *     a uniformly random division of the N ids into consecutive batches of a
 *     random permutation, batch size p, the last batch of size N mod p when p
 *     does not divide N; in-batch interaction scaled by 1/(|C|-1), zero for a
 *     singleton batch; one explicit Euler-Maruyama step from the old positions
 *     (Sec. 4.1 solves each step by forward Euler).
 *   - the random permutation (Sec. 2.1 takes any uniform shuffle): ids sorted
 *     ascending by a 64-bit counter-based Philox4x32-10 key, ties broken by id.
 *   - Brownian increments (Sec. 3, eq. "coupling"): indexed by particle id and
 *     step, never by batch slot, so RBM and the direct step see the same
 *     B^i(t_m) - B^i(t_{m-1}) (the paper's synchronous coupling).
 *   - K(0) := 0 for every kernel (the paper never evaluates K at coincident
 *     points; singular kernels are undefined there).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "rbm_oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11).  One round maps (c0,c1,c2,c3) with key (k0,k1)  */
/* to (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0)); the key is   */
/* advanced by the Weyl constants between rounds.                            */
/* ------------------------------------------------------------------------ */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    memcpy(out, c, sizeof(c));
}

/* Counter layout: (particle id, step m mod 2^32, replica r, stream*256+call),
 * key = (seed low word, seed high word). */
static void orc_draw(uint64_t seed, uint32_t id, int64_t m, uint32_t r,
                     uint32_t stream, uint32_t call, uint32_t out[4])
{
    uint32_t ctr[4] = {id, (uint32_t)(uint64_t)m, r, stream * 256u + call};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Random division (Sec. 2.1): permutation keys and the sorted permutation.  */
/* ------------------------------------------------------------------------ */
void orc_perm_keys(const orc_params *prm, int64_t m, uint64_t *keys)
{
    for (int64_t i = 0; i < prm->n; ++i) {
        uint32_t w[4];
        orc_draw(prm->seed, (uint32_t)i, m, prm->replica, ORC_STREAM_PERM, 0, w);
        keys[i] = ((uint64_t)w[1] << 32) | (uint64_t)w[0];
    }
}

typedef struct { uint64_t key; uint32_t id; } orc_keyed;

static int orc_keyed_cmp(const void *a, const void *b)
{
    const orc_keyed *x = (const orc_keyed *)a, *y = (const orc_keyed *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

void orc_permutation(const orc_params *prm, int64_t m, uint32_t *perm)
{
    int64_t n = prm->n;
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    orc_keyed *rec = (orc_keyed *)malloc(sizeof(orc_keyed) * (size_t)n);
    orc_perm_keys(prm, m, keys);
    for (int64_t i = 0; i < n; ++i) { rec[i].key = keys[i]; rec[i].id = (uint32_t)i; }
    qsort(rec, (size_t)n, sizeof(orc_keyed), orc_keyed_cmp);
    for (int64_t i = 0; i < n; ++i) perm[i] = rec[i].id;
    free(rec);
    free(keys);
}

/* ------------------------------------------------------------------------ */
/* Brownian increments: Box-Muller on Philox uniforms.                       */
/* Pair t = 0 .. ceil(d/2)-1 takes two uniforms u = (top b bits + 1) 2^-b in  */
/* (0, 1] (b = 53 for FP64 runs, 24 for FP32 runs; see orc_pair_uniforms for  */
/* which words of which draw), and                                            */
/* z_{2t} = sqrt(-2 ln u1) cos(2 pi u2), z_{2t+1} = sqrt(-2 ln u1) sin(2 pi u2)*/
/* ------------------------------------------------------------------------ */
static double orc_uniform(uint32_t lo, uint32_t hi, int bits)
{
    uint64_t w = ((uint64_t)hi << 32) | (uint64_t)lo;
    uint64_t top = w >> (64 - bits);
    return ldexp((double)(top + 1u), -bits);
}

/* The standard normal vector of particle id for the step with index m of a  */
/* run with step dt (one Box-Muller draw per pair of coordinates).           */
/* Uniform inputs of Box-Muller pair t.  53-bit runs: draw t, the 64-bit    */
/* words a1:a0 and a3:a2.  24-bit runs: one 32-bit word per uniform, so one   */
/* draw (call t/2) serves two pairs: even t the words a1, a3 (the same top 24 */
/* bits the 64-bit reading takes), odd t the words a0, a2.                    */
static void orc_pair_uniforms(const orc_params *prm, uint32_t id, int64_t m, int t, double *u1, double *u2)
{
    uint32_t a[4];
    if (prm->ubits == 24) {
        orc_draw(prm->seed, id, m, prm->replica, ORC_STREAM_NOISE, (uint32_t)(t / 2), a);
        uint32_t w1 = (t % 2 == 0) ? a[1] : a[0];
        uint32_t w2 = (t % 2 == 0) ? a[3] : a[2];
        *u1 = orc_uniform(0u, w1, 24);
        *u2 = orc_uniform(0u, w2, 24);
        return;
    }
    orc_draw(prm->seed, id, m, prm->replica, ORC_STREAM_NOISE, (uint32_t)t, a);
    *u1 = orc_uniform(a[0], a[1], prm->ubits);
    *u2 = orc_uniform(a[2], a[3], prm->ubits);
}

static void orc_normals_plain(const orc_params *prm, uint32_t id, int64_t m, double *z)
{
    int d = prm->d;
    for (int t = 0; 2 * t < d; ++t) {
        double u1, u2;
        orc_pair_uniforms(prm, id, m, t, &u1, &u2);
        double rad = sqrt(-2.0 * log(u1));
        double ang = 2.0 * M_PI * u2;
        z[2 * t] = rad * cos(ang);
        if (2 * t + 1 < d) z[2 * t + 1] = rad * sin(ang);
    }
}

/* Path coupling across step sizes (the synchronous coupling of Sec. 3, eq.   */
/* "coupling": the compared processes are driven by the same Brownian motion  */
/* B^i).  A run with step dt and refinement r draws the increment of its step */
/* m, B^i(t_{m+1}) - B^i(t_m) = sqrt(dt) z, as the sum of the r increments     */
/* sqrt(dt/r) z_k that a run with step dt/r draws over the same interval,      */
/* fine steps m r + k, k = 0..r-1:  z = r^(-1/2) sum_k z_k.  With r = 1 it is  */
/* the plain draw.  (The paper compares each method with a fine-step direct    */
/* reference, Sec. 4.1; this makes every step size see one Brownian path.)     */
void orc_normals_one(const orc_params *prm, uint32_t id, int64_t m, double *z)
{
    int d = prm->d;
    int64_t r = prm->noise_refine > 1 ? prm->noise_refine : 1;
    if (r == 1) {
        orc_normals_plain(prm, id, m, z);
        return;
    }
    double sum[3] = {0.0, 0.0, 0.0}, zk[4];
    for (int64_t k = 0; k < r; ++k) {
        orc_normals_plain(prm, id, m * r + k, zk);
        for (int c = 0; c < d; ++c) sum[c] += zk[c];
    }
    for (int c = 0; c < d; ++c) z[c] = sum[c] / sqrt((double)r);
}

void orc_normals(const orc_params *prm, int64_t m, double *z)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < prm->n; ++i) orc_normals_one(prm, (uint32_t)i, m, z + i * prm->d);
}

/* ------------------------------------------------------------------------ */
/* Interaction kernels K and confining potentials V.                         */
/* ------------------------------------------------------------------------ */

/* Squared norm used for every decision a kernel takes (coincidence, cut-off
 * radius).  When the run under test computes in FP32, the decision is taken
 * on the FP32 value evaluated as fma(dz,dz, fma(dy,dy, dx*dx)) of FP32
 * differences, so both sides take it in the same precision. */
static double orc_decision_r2(const orc_params *prm, const double *xi, const double *xj)
{
    int d = prm->d;
    if (prm->decide_f32) {
        float r2 = 0.0f;
        for (int k = 0; k < d; ++k) {
            float dx = (float)xi[k] - (float)xj[k];
            r2 = (k == 0) ? dx * dx : fmaf(dx, dx, r2);
        }
        return (double)r2;
    }
    double r2 = 0.0;
    for (int k = 0; k < d; ++k) {
        double dx = xi[k] - xj[k];
        r2 = (k == 0) ? dx * dx : fma(dx, dx, r2);
    }
    return r2;
}

/* out = K(xi - xj), x = xi - xj. */
void orc_kernel_pair(const orc_params *prm, const double *xi, const double *xj, double *out)
{
    int d = prm->d;
    double x[3] = {0.0, 0.0, 0.0};
    double r2 = 0.0;                                    /* |x|^2 */
    for (int k = 0; k < d; ++k) { x[k] = xi[k] - xj[k]; r2 += x[k] * x[k]; }
    double r2_decide = orc_decision_r2(prm, xi, xj);
    double radius_sq = prm->k_param * prm->k_param;
    if (prm->decide_f32) radius_sq = (double)(float)radius_sq;
    for (int k = 0; k < d; ++k) out[k] = 0.0;
    if (r2_decide == 0.0) return;                       /* K(0) := 0 */
    for (int k = 0; k < d; ++k) {
        switch (prm->k_kind) {
        case ORC_K_INV1D:        out[k] = 1.0 / x[k]; break;                        /* 1/x            */
        case ORC_K_COULOMB:      out[k] = x[k] / (r2 * sqrt(r2)); break;            /* x/|x|^3        */
        case ORC_K_BOUNDED_CONF: out[k] = (r2_decide < radius_sq) ? -x[k] : 0.0; break; /* -x 1{|x|<R} */
        case ORC_K_GAUSS_AGG:    out[k] = -x[k] * exp(-0.5 * r2); break;            /* -x e^{-|x|^2/2} */
        case ORC_K_REG_ATTRACT:  out[k] = -x[k] / (r2 + prm->k_param); break;       /* -x/(|x|^2+eps) */
        case ORC_K_SMOOTH_TEST:  out[k] = x[k] / (1.0 + r2); break;                 /* x/(1+|x|^2)    */
        case ORC_K_LINEAR:       out[k] = -prm->k_param * x[k]; break;              /* -c x           */
        default:                 out[k] = 0.0; break;
        }
    }
}

/* out = -grad V(x). */
static void orc_confining(const orc_params *prm, const double *x, double *out)
{
    for (int k = 0; k < prm->d; ++k)
        out[k] = (prm->v_kind == ORC_V_QUADRATIC) ? -prm->v_coef * x[k] : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Interaction forces.                                                       */
/* ------------------------------------------------------------------------ */

/* Direct: FK_i = 1/(N-1) sum_{j != i, ascending j} K(X^i - X^j)   (Sec. 1). */
static void orc_direct_interaction_one(const orc_params *prm, const double *X, int64_t i, double *fk)
{
    int d = prm->d;
    double acc[3] = {0.0, 0.0, 0.0}, kij[3];
    for (int64_t j = 0; j < prm->n; ++j) {
        if (j == i) continue;
        orc_kernel_pair(prm, X + i * d, X + j * d, kij);
        for (int k = 0; k < d; ++k) acc[k] += kij[k];
    }
    for (int k = 0; k < d; ++k) fk[k] = acc[k] / (double)(prm->n - 1);
}

void orc_direct_interaction(const orc_params *prm, const double *X, double *FK)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < prm->n; ++i) orc_direct_interaction_one(prm, X, i, FK + i * prm->d);
}

static int orc_u32_cmp(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

/* RBM-1 (eq. "firstalgorithm"): for i in batch C_q,
 * FK_i = 1/(|C_q|-1) sum_{j in C_q, j != i, ascending j} K(X^i - X^j); 0 if |C_q| = 1.
 * Batch q is perm[q p .. min((q+1) p, N) - 1]. */
void orc_rbm_interaction(const orc_params *prm, const double *X, const uint32_t *perm, double *FK)
{
    int64_t n = prm->n, p = prm->p;
    int d = prm->d;
    int64_t nbatch = (n + p - 1) / p;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < nbatch; ++q) {
        int64_t lo = q * p, hi = (q + 1) * p < n ? (q + 1) * p : n;
        int64_t sz = hi - lo;
        uint32_t *members = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)sz);
        memcpy(members, perm + lo, sizeof(uint32_t) * (size_t)sz);
        qsort(members, (size_t)sz, sizeof(uint32_t), orc_u32_cmp);
        for (int64_t a = 0; a < sz; ++a) {
            int64_t i = members[a];
            double acc[3] = {0.0, 0.0, 0.0}, kij[3];
            for (int64_t b = 0; b < sz; ++b) {
                int64_t j = members[b];
                if (j == i) continue;
                orc_kernel_pair(prm, X + i * d, X + j * d, kij);
                for (int k = 0; k < d; ++k) acc[k] += kij[k];
            }
            for (int k = 0; k < d; ++k) FK[i * d + k] = (sz > 1) ? acc[k] / (double)(sz - 1) : 0.0;
        }
        free(members);
    }
}

/* ------------------------------------------------------------------------ */
/* Euler-Maruyama update from a given interaction force (Sec. 4.1: forward    */
/* Euler per step; the Thomson runs project back to the sphere, Sec. 5.1).   */
/*   X'^i = X^i + dt (FK_i - grad V(X^i)) + sigma sqrt(dt) z_i               */
/*   RENORM: X'^i <- X'^i / |X'^i|                                           */
/* ------------------------------------------------------------------------ */
/* With multiplicative noise (gbm = 1, the wealth model of Sec. 5.2, eq.     */
/* "wealth": sigma X dB) the noise term is sigma sqrt(tau) x z in the Euler-  */
/* Maruyama step; after the exact pair flow of the splitting scheme the noise */
/* sub-step is the exact geometric Brownian flow x exp(-sigma^2 tau/2 +       */
/* sigma sqrt(tau) z) (Ito), which keeps the expected wealth.                 */
static void orc_euler_update_one(const orc_params *prm, uint32_t id, const double *x, const double *fk, int64_t m,
                                 double *y, int split_flow)
{
    int d = prm->d;
    double sq = prm->sigma * sqrt(prm->dt);
    double z[4] = {0.0, 0.0, 0.0, 0.0}, fv[3];
    orc_normals_one(prm, id, m, z);
    orc_confining(prm, x, fv);
    for (int k = 0; k < d; ++k) {
        if (!prm->gbm)      y[k] = x[k] + prm->dt * (fk[k] + fv[k]) + sq * z[k];
        else if (split_flow) y[k] = x[k] * exp(-0.5 * sq * sq + sq * z[k]) + prm->dt * (fk[k] + fv[k]);
        else                y[k] = x[k] + prm->dt * (fk[k] + fv[k]) + sq * x[k] * z[k];
    }
    if (prm->renorm) {
        double nrm = 0.0;
        for (int k = 0; k < d; ++k) nrm += y[k] * y[k];
        nrm = sqrt(nrm);
        for (int k = 0; k < d; ++k) y[k] /= nrm;
    }
}

static void orc_update_all(const orc_params *prm, double *X, const double *FK, int64_t m, int split_flow)
{
    int d = prm->d;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < prm->n; ++i) {
        double y[3];
        orc_euler_update_one(prm, (uint32_t)i, X + i * d, FK + i * d, m, y, split_flow);
        for (int k = 0; k < d; ++k) X[i * d + k] = y[k];
    }
}

void orc_euler_update(const orc_params *prm, double *X, const double *FK, int64_t m)
{
    orc_update_all(prm, X, FK, m, 0);
}

/* ------------------------------------------------------------------------ */
/* Splitting scheme for singular kernels, p = 2 (Sec. 2.3 item 5; used for   */
/* the Dyson Brownian motion in Sec. 4.2 and the Thomson problem in Sec. 5.1).*/
/* Sub-step 1 solves the pair interaction dX^i = K(X^i - X^j) dt exactly over */
/* [0, tau]; sub-step 2 is the Euler-Maruyama step of -grad V and the noise,  */
/* taken from the sub-step-1 positions Y.                                     */
/*   K = 1/x (d = 1): delta = X^i - X^j obeys d(delta^2)/dt = 4, so           */
/*     Y^i,j = (X^i + X^j)/2 +- sgn(delta) sqrt(delta^2 + 4 tau) / 2.         */
/*   K = x/|x|^3: the direction of delta is fixed and d|delta|^3/dt = 6, so   */
/*     Y^i,j = (X^i + X^j)/2 +- (delta/|delta|) (|delta|^3 + 6 tau)^(1/3) / 2.*/
/*   K = -c x (the wealth model's quadratic trading, Sec. 5.2): d delta/dt =  */
/*     -2 c delta, so delta shrinks by exp(-2 c tau) about the fixed mean.    */
/* (The paper prints both formulas without the factors 1/2; the ODE fixes    */
/* them.)  A singleton batch and a coincident pair (delta = 0, K(0) = 0) keep */
/* Y = X.                                                                     */
/* ------------------------------------------------------------------------ */
void orc_split_pair_solve(const orc_params *prm, const double *xi, const double *xj, double *yi, double *yj)
{
    int d = prm->d;
    double delta[3] = {0.0, 0.0, 0.0}, mid[3] = {0.0, 0.0, 0.0}, len2 = 0.0;
    for (int k = 0; k < d; ++k) {
        delta[k] = xi[k] - xj[k];
        mid[k] = 0.5 * (xi[k] + xj[k]);
        len2 += delta[k] * delta[k];
    }
    if (orc_decision_r2(prm, xi, xj) == 0.0) {
        for (int k = 0; k < d; ++k) { yi[k] = xi[k]; yj[k] = xj[k]; }
        return;
    }
    double len = sqrt(len2), newlen;
    if (prm->k_kind == ORC_K_INV1D)       newlen = sqrt(len2 + 4.0 * prm->dt);
    else if (prm->k_kind == ORC_K_LINEAR) newlen = len * exp(-2.0 * prm->k_param * prm->dt);
    else                                  newlen = cbrt(len2 * len + 6.0 * prm->dt);
    for (int k = 0; k < d; ++k) {
        double half = 0.5 * newlen * (delta[k] / len);
        yi[k] = mid[k] + half;
        yj[k] = mid[k] - half;
    }
}

void orc_rbm_split_step(const orc_params *prm, double *X, int64_t m)
{
    int64_t n = prm->n;
    int d = prm->d;
    uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    double *Y = (double *)malloc(sizeof(double) * (size_t)n * (size_t)d);
    double *zero = (double *)calloc((size_t)n * (size_t)d, sizeof(double));
    orc_permutation(prm, m, perm);
    memcpy(Y, X, sizeof(double) * (size_t)n * (size_t)d);
    for (int64_t q = 0; 2 * q + 1 < n; ++q) {
        uint32_t i = perm[2 * q], j = perm[2 * q + 1];
        if (j < i) { uint32_t t = i; i = j; j = t; }   /* smaller id first */
        orc_split_pair_solve(prm, X + (int64_t)i * d, X + (int64_t)j * d, Y + (int64_t)i * d, Y + (int64_t)j * d);
    }
    orc_update_all(prm, Y, zero, m, 1);              /* -grad V(Y), noise, renorm */
    memcpy(X, Y, sizeof(double) * (size_t)n * (size_t)d);
    free(zero);
    free(Y);
    free(perm);
}

/* One RBM-1 step m -> m+1, in place (Algorithm "randomdiv"). */
void orc_rbm_step(const orc_params *prm, double *X, int64_t m)
{
    size_t nd = (size_t)prm->n * (size_t)prm->d;
    uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)prm->n);
    double *FK = (double *)malloc(sizeof(double) * nd);
    orc_permutation(prm, m, perm);
    orc_rbm_interaction(prm, X, perm, FK);
    orc_euler_update(prm, X, FK, m);
    free(FK);
    free(perm);
}

/* One direct forward-Euler step m -> m+1 with the same Brownian increments. */
void orc_direct_step(const orc_params *prm, double *X, int64_t m)
{
    size_t nd = (size_t)prm->n * (size_t)prm->d;
    double *FK = (double *)malloc(sizeof(double) * nd);
    orc_direct_interaction(prm, X, FK);
    orc_euler_update(prm, X, FK, m);
    free(FK);
}

/* ------------------------------------------------------------------------ */
/* Second-order (Hamiltonian) system of Appendix A, eq. "Hamil1":            */
/*   dX/dt = V,  dV/dt = b(X) + 1/(N-1) sum_j K(X^i - X^j),  b = -grad V,    */
/* integrated by the Verlet scheme of Sec. 4.1 (end):                         */
/*   X_1 = X_0 + tau V_0 + tau^2 F_0 / 2,                                    */
/*   X_{n+1} = 2 X_n - X_{n-1} + tau^2 F_n,  n >= 1,                          */
/* F_n = b(X_n) + the interaction of step n: the in-batch sum of RBM-1        */
/* (eq. "Hamilrand", the random division of step n) or the full sum.          */
/* P holds V_0 before the first step (first = 1) and X_{n-1} afterwards; the */
/* step writes X_{n+1} to X and X_n to P.  No noise.                          */
/* ------------------------------------------------------------------------ */
static void orc_verlet_update(const orc_params *prm, double *X, double *P, const double *FK, int first)
{
    int d = prm->d;
    double tau = prm->dt;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < prm->n; ++i) {
        double fv[3];
        orc_confining(prm, X + i * d, fv);
        for (int k = 0; k < d; ++k) {
            double x = X[i * d + k], q = P[i * d + k], f = FK[i * d + k] + fv[k];
            double y = first ? x + tau * q + 0.5 * tau * tau * f : 2.0 * x - q + tau * tau * f;
            P[i * d + k] = x;
            X[i * d + k] = y;
        }
    }
}

void orc_rbm_verlet_step(const orc_params *prm, double *X, double *P, int64_t m, int first)
{
    size_t nd = (size_t)prm->n * (size_t)prm->d;
    uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)prm->n);
    double *FK = (double *)malloc(sizeof(double) * nd);
    orc_permutation(prm, m, perm);
    orc_rbm_interaction(prm, X, perm, FK);
    orc_verlet_update(prm, X, P, FK, first);
    free(FK);
    free(perm);
}

void orc_direct_verlet_step(const orc_params *prm, double *X, double *P, int first)
{
    size_t nd = (size_t)prm->n * (size_t)prm->d;
    double *FK = (double *)malloc(sizeof(double) * nd);
    orc_direct_interaction(prm, X, FK);
    orc_verlet_update(prm, X, P, FK, first);
    free(FK);
}

/* ------------------------------------------------------------------------ */
/* RBM-r (Sec. 2.2, Algorithm "fullyrandom"): iteration k picks a set C of p  */
/* distinct particles at random and moves its members by one Euler-Maruyama   */
/* step of size tau of the p-particle system of eq. "secondalgB", every force */
/* taken from the positions before the iteration; iterations run strictly in */
/* order, each seeing the positions the previous ones left.  floor(N/p)       */
/* iterations (at least one) carry the pseudo-time of one RBM-1 step, as the  */
/* paper's RBM-r' form (Algorithm "randomreplacement") spells out.            */
/* Readings (the paper says only "randomly"):                                */
/*   - the set: the words w0..w3 of the Philox blocks at counters             */
/*     (k mod 2^32, k div 2^32, r, 7*256 + c), c = 0, 1, ..., 255, in order,  */
/*     each mapped to the id floor(w N / 2^32); an id already taken is        */
/*     skipped; the first p distinct ids, in the order drawn, are the slots   */
/*     0..p-1 (the smallest ids not yet taken fill any slot still empty after */
/*     1024 words, which needs p close to N and never happens for p <= 32);   */
/*   - the noise of slot s: Box-Muller as for RBM-1 from the blocks at        */
/*     counters (k mod 2^32, k div 2^32, r, 8*256 + 2 s + t), t < ceil(d/2);  */
/*   - the in-set sum runs over the other slots in slot order.               */
/* ------------------------------------------------------------------------ */
#define ORC_STREAM_RBMR_SET 7u
#define ORC_STREAM_RBMR_NOISE 8u

int64_t orc_rbmr_iterations_per_step(const orc_params *prm)
{
    int64_t k = prm->n / prm->p;
    return k > 0 ? k : 1;
}

void orc_rbmr_set(const orc_params *prm, int64_t k, uint32_t *set)
{
    uint32_t key[2] = {(uint32_t)prm->seed, (uint32_t)(prm->seed >> 32)};
    int p = prm->p, got = 0;
    for (uint32_t c = 0; c < 256u && got < p; ++c) {
        uint32_t ctr[4] = {(uint32_t)(uint64_t)k, (uint32_t)((uint64_t)k >> 32), prm->replica,
                           ORC_STREAM_RBMR_SET * 256u + c};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        for (int q = 0; q < 4 && got < p; ++q) {
            uint32_t id = (uint32_t)(((uint64_t)w[q] * (uint64_t)prm->n) >> 32);
            int taken = 0;
            for (int s = 0; s < got; ++s) taken |= (set[s] == id);
            if (!taken) set[got++] = id;
        }
    }
    for (uint32_t id = 0; got < p; ++id) {
        int taken = 0;
        for (int s = 0; s < got; ++s) taken |= (set[s] == id);
        if (!taken) set[got++] = id;
    }
}

static void orc_rbmr_normals(const orc_params *prm, int64_t k, int slot, double *z)
{
    uint32_t key[2] = {(uint32_t)prm->seed, (uint32_t)(prm->seed >> 32)};
    for (int t = 0; 2 * t < prm->d; ++t) {
        uint32_t ctr[4] = {(uint32_t)(uint64_t)k, (uint32_t)((uint64_t)k >> 32), prm->replica,
                           ORC_STREAM_RBMR_NOISE * 256u + 2u * (uint32_t)slot + (uint32_t)t};
        uint32_t a[4];
        orc_philox4x32_10(ctr, key, a);
        double u1 = orc_uniform(a[0], a[1], prm->ubits);
        double u2 = orc_uniform(a[2], a[3], prm->ubits);
        double rad = sqrt(-2.0 * log(u1));
        double ang = 2.0 * M_PI * u2;
        z[2 * t] = rad * cos(ang);
        if (2 * t + 1 < prm->d) z[2 * t + 1] = rad * sin(ang);
    }
}

void orc_rbmr_iteration(const orc_params *prm, double *X, int64_t k)
{
    int p = prm->p, d = prm->d;
    uint32_t *set = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)p);
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)p);
    orc_rbmr_set(prm, k, set);
    for (int s = 0; s < p; ++s) {
        double acc[3] = {0.0, 0.0, 0.0}, kst[3];
        for (int t = 0; t < p; ++t) {
            if (t == s) continue;
            orc_kernel_pair(prm, X + (size_t)set[s] * d, X + (size_t)set[t] * d, kst);
            for (int c = 0; c < d; ++c) acc[c] += kst[c];
        }
        for (int c = 0; c < d; ++c) F[3 * s + c] = acc[c] / (double)(p - 1);
    }
    double sq = prm->sigma * sqrt(prm->dt);
    for (int s = 0; s < p; ++s) {
        double *x = X + (size_t)set[s] * d;
        double z[4] = {0.0, 0.0, 0.0, 0.0}, fv[3], y[3];
        orc_rbmr_normals(prm, k, s, z);
        orc_confining(prm, x, fv);
        for (int c = 0; c < d; ++c) y[c] = x[c] + prm->dt * (F[3 * s + c] + fv[c]) + sq * z[c];
        if (prm->renorm) {
            double nrm = 0.0;
            for (int c = 0; c < d; ++c) nrm += y[c] * y[c];
            nrm = sqrt(nrm);
            for (int c = 0; c < d; ++c) y[c] /= nrm;
        }
        for (int c = 0; c < d; ++c) x[c] = y[c];
    }
    free(F);
    free(set);
}

/* One RBM-r step m -> m+1: iterations m K .. m K + K - 1, K = floor(N/p). */
void orc_rbmr_step(const orc_params *prm, double *X, int64_t m)
{
    int64_t K = orc_rbmr_iterations_per_step(prm);
    for (int64_t j = 0; j < K; ++j) orc_rbmr_iteration(prm, X, m * K + j);
}

/* The direct step of the listed particles only: Y[a] = new position of
 * particle idx[a] after one direct step from X (same arithmetic as
 * orc_direct_step, restricted to a sample so large N stays affordable). */
void orc_direct_step_sampled(const orc_params *prm, const double *X, int64_t m, const int64_t *idx, int64_t nidx,
                             double *Y)
{
    int d = prm->d;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t a = 0; a < nidx; ++a) {
        double fk[3];
        int64_t i = idx[a];
        orc_direct_interaction_one(prm, X, i, fk);
        orc_euler_update_one(prm, (uint32_t)i, X + i * d, fk, m, Y + a * d, 0);
    }
}

/* Mean-field force at query points: F(q) = 1/(N-1) sum_j K(q - X^j) over all
 * N particles (the direct sum of Sec. 1 evaluated at an arbitrary point;
 * a query that coincides with a particle gets K(0) = 0 from it). */
void orc_direct_forces_at(const orc_params *prm, const double *X, const double *Q, int64_t nq, double *F)
{
    int d = prm->d;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t a = 0; a < nq; ++a) {
        double acc[3] = {0.0, 0.0, 0.0}, kij[3];
        for (int64_t j = 0; j < prm->n; ++j) {
            orc_kernel_pair(prm, Q + a * d, X + j * d, kij);
            for (int k = 0; k < d; ++k) acc[k] += kij[k];
        }
        for (int k = 0; k < d; ++k) F[a * d + k] = acc[k] / (double)(prm->n - 1);
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
