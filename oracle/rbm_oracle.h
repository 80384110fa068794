/*
 * Plain FP64 CPU oracle of RBM-1 and of the direct step (arXiv:1812.10575).
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark; never by the product path.  This header
 * belongs to the oracle alone and shares nothing with the CUDA library.
 *
 * Positions are N x d row-major doubles (no padding).
 */
#ifndef RBM_ORACLE_H
#define RBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_V_ZERO = 0, ORC_V_QUADRATIC = 1 };
enum {
    ORC_K_INV1D = 0,        /* K(x) = 1/x, d = 1 (Dyson Brownian motion, Sec. 4.2) */
    ORC_K_COULOMB = 1,      /* K(x) = x/|x|^3 (Thomson problem, Sec. 5.1)          */
    ORC_K_BOUNDED_CONF = 2, /* K(x) = -x 1{|x| < R}, R = k_param (opinions, Sec. 5.2) */
    ORC_K_GAUSS_AGG = 3,    /* K(x) = -x exp(-|x|^2/2)                             */
    ORC_K_REG_ATTRACT = 4,  /* K(x) = -x/(|x|^2 + eps), eps = k_param              */
    ORC_K_SMOOTH_TEST = 5,  /* K(x) = x/(1+|x|^2) (Sec. 4.1 test example)          */
    ORC_K_LINEAR = 6        /* K(x) = -c x, c = k_param                            */
};
enum { ORC_STREAM_PERM = 0, ORC_STREAM_NOISE = 1 };

typedef struct {
    int64_t n;        /* particles N                                        */
    int32_t d;        /* dimension, 1..3                                    */
    int32_t p;        /* batch size                                         */
    double dt;        /* time step tau                                      */
    double sigma;     /* noise amplitude                                    */
    uint64_t seed;    /* Philox key                                         */
    int32_t v_kind;   /* ORC_V_*                                            */
    int32_t k_kind;   /* ORC_K_*                                            */
    double v_coef;    /* V = v_coef |x|^2 / 2                               */
    double k_param;   /* kernel parameter (R, eps or c)                     */
    int32_t renorm;   /* 1: project onto the unit sphere after each step    */
    int32_t ubits;    /* uniform bits per Box-Muller input: 53 or 24        */
    int32_t decide_f32; /* 1: kernel decisions on the FP32 squared norm     */
    uint32_t replica; /* replica index r (third counter word)               */
    int32_t gbm;      /* 1: multiplicative noise sigma X dB (wealth model)  */
    int32_t noise_refine; /* r >= 1 (0 reads as 1): the increment of step m  */
                      /* is the normalised sum of the r increments of a   */
                      /* run with step dt/r over the same interval         */
} orc_params;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_perm_keys(const orc_params *prm, int64_t m, uint64_t *keys);
void orc_permutation(const orc_params *prm, int64_t m, uint32_t *perm);
void orc_normals_one(const orc_params *prm, uint32_t id, int64_t m, double *z);
void orc_normals(const orc_params *prm, int64_t m, double *z);
void orc_kernel_pair(const orc_params *prm, const double *xi, const double *xj, double *out);
void orc_direct_interaction(const orc_params *prm, const double *X, double *FK);
void orc_rbm_interaction(const orc_params *prm, const double *X, const uint32_t *perm, double *FK);
void orc_euler_update(const orc_params *prm, double *X, const double *FK, int64_t m);
void orc_split_pair_solve(const orc_params *prm, const double *xi, const double *xj, double *yi, double *yj);
void orc_rbm_split_step(const orc_params *prm, double *X, int64_t m);
void orc_rbm_step(const orc_params *prm, double *X, int64_t m);
void orc_direct_step(const orc_params *prm, double *X, int64_t m);
void orc_direct_step_sampled(const orc_params *prm, const double *X, int64_t m, const int64_t *idx, int64_t nidx,
                             double *Y);
void orc_direct_forces_at(const orc_params *prm, const double *X, const double *Q, int64_t nq, double *F);
void orc_rbm_verlet_step(const orc_params *prm, double *X, double *P, int64_t m, int first);
void orc_direct_verlet_step(const orc_params *prm, double *X, double *P, int first);
int64_t orc_rbmr_iterations_per_step(const orc_params *prm);
void orc_rbmr_set(const orc_params *prm, int64_t k, uint32_t *set);
void orc_rbmr_iteration(const orc_params *prm, double *X, int64_t k);
void orc_rbmr_step(const orc_params *prm, double *X, int64_t m);
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
