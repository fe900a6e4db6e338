/* pcpm_warmstart.h - learned warm start for PCPM PageRank (C ABI).
 *
 * Not in the paper. PageRank by power iteration (Eq. 1) normally starts from
 * the uniform vector 1/n. A small per-node network predicts log(n * PR*(v))
 * from cheap features of the graph, and the iteration starts from the
 * softmax of the prediction (pcpm_pagerank's pr_init) instead; it converges to
 * the same fixed point, and the plain uniform start stays the reference.
 *
 * Features of node v, PCPM_WS_FEATURES = 5, row-major float[n][5]:
 *   0  log1p(indeg(v))
 *   1  log1p(outdeg(v))
 *   2  log1p(sum of indeg(u) over in-neighbours u)
 *   3  log1p(sum of outdeg(u) over in-neighbours u)
 * The in-degree and both sums are exact unsigned 32-bit in-edge sums over the
 * handle's bins (pcpm_ws_degree_sums); the logarithms are FP32 (log1pf of the
 * count converted to float).
 *   4  log(n * PR_1(v)), PR_1 one Eq. 1 step from the uniform start on the
 *      handle (d = 0.85, dangling mass spread uniformly)
 * Network: standardise x^ = (x - mu) * inv_sigma; h1 = relu(W1 x^ + b1);
 * h2 = relu(W2 h1 + b2); y = w3 . h2 + b3 (width PCPM_WS_HIDDEN = 64).
 * Parameters: one float array of PCPM_WS_PARAMS entries, in this order:
 *   mu[5], inv_sigma[5], W1[64][5], b1[64], W2[64][64], b2[64], w3[64], b3.
 * mu and inv_sigma are set by the caller and not trained.
 *
 * All pointers are device memory unless stated; every call is enqueued on
 * `stream` and returns PCPM_* status codes of pcpm.h.
 */
#ifndef PCPM_WARMSTART_H
#define PCPM_WARMSTART_H

#include <stdint.h>

#include "pcpm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PCPM_WS_FEATURES 5
#define PCPM_WS_HIDDEN 64
#define PCPM_WS_PARAMS (2 * 5 + 64 * 5 + 64 + 64 * 64 + 64 + 64 + 1)
/* first trainable entry (W1) */
#define PCPM_WS_TRAINABLE_OFFSET 10

/* Features of every node of the graph the handle was built from.
 *   row_ptr, col  the device CSR given to pcpm_build (uint32[n+1], uint32[m];
 *                 col is not read: the sums come from the handle's bins).
 *   features      float[n][5], written.
 * Runs the three exact sums of pcpm_ws_degree_sums, then one iteration for
 * PR_1, and leaves the handle's solver state after PR_1. Allocates 16 bytes per
 * node of stream-ordered device scratch and frees it. Synchronises.
 * PCPM_EINVAL for a destination shard (pcpm_build_shard). */
int pcpm_ws_features(pcpm_png* png, const uint32_t* row_ptr, const uint32_t* col, float* features,
                     void* stream);

/* The integer parts of features 0, 2 and 3, exactly: sums (uint32[3][n]) gets
 * indeg(v), the sum of indeg(u) and the sum of outdeg(u) over the in-edges
 * u -> v, each one pass over the handle's canonical bins (every in-edge of a
 * node of partition p lies in bin p; Sec. 3.1) with unsigned 32-bit
 * shared-memory sums per bin. The source of each destination ID is that of its
 * update (Algorithm 4's update index). On handles with FP32 update bins the
 * per-source degrees are first scattered into the bins (Algorithm 3, copied
 * bit for bit), so the sums read them in bin order instead of at random. The
 * in-degree comes from the build where the window layout kept it. Overwrites
 * the handle's update bins and solver state (pcpm_reset before solving).
 * row_ptr: the CSR given to pcpm_build. Synchronises;
 * PCPM_EDEVICE if a sum passes 2^32 - 1. */
int pcpm_ws_degree_sums(pcpm_png* png, const uint32_t* row_ptr, uint32_t* sums, void* stream);

/* Feature statistics for the standardisation, summed in FP64 over all n rows
 * and added to moments (double[11]: rows, then the sum of each column, then
 * the sum of squares of each column); zero it before the first graph.
 * pcpm_ws_standardisation writes params[0..10): mu = the mean and inv_sigma =
 * 1 / max(population standard deviation, 1e-6) of each column. */
int pcpm_ws_feature_moments(const float* features, uint32_t n, double* moments, void* stream);
int pcpm_ws_standardisation(const double* moments, float* params, void* stream);

/* Training targets: target(v) = log(n * pr(v)) computed in FP64 and rounded
 * to float, for ranks pr (float[n], positive) of a graph of n nodes. */
int pcpm_ws_targets(const float* pr, uint32_t n, float* target, void* stream);

/* Network output for n feature rows, with W1, b1, W2, b2, w3, b3 rounded to
 * bfloat16 (nearest even). Both hidden layers run on the tensor cores (mma
 * m16n8k16, BF16 operands, FP32 accumulation) with the standardised inputs
 * and h1 rounded to BF16 (relative error <= 2^-9 each); the standardisation,
 * biases, ReLU and the output dot product with w3 are FP32.
 *   params float[PCPM_WS_PARAMS]; features float[n][5]; out float[n]. */
int pcpm_ws_predict(const float* params, const float* features, uint32_t n, float* out, void* stream);

/* Mean-squared-error loss L = sum_v (y(v) - target(v))^2 / n over n rows, with
 * FP32 weights, and its gradient.
 *   grad  float[PCPM_WS_PARAMS]: zeroed by the call, then dL/dparams (0 for
 *         mu and inv_sigma).
 *   loss  double[1]: written.
 * FP32 arithmetic; per-tile sums of the gradient are added with atomics, so
 * the last bits depend on the order. */
int pcpm_ws_loss_grad(const float* params, const float* features, const float* target, uint32_t n,
                      float* grad, double* loss, void* stream);

/* One Adam step (Kingma and Ba, 2015) on the trainable entries, step >= 1.
 *   m, v  float[PCPM_WS_PARAMS] first and second moments, updated in place. */
int pcpm_ws_adam(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1,
                 float beta2, float eps, void* stream);

/* Initial ranks from predictions: pr(v) = exp(p(v)) / sum_u exp(p(u)) with
 * p = pred clamped to [-80, 80] (so no term overflows FP32), the sum in FP64,
 * each quotient as expf(p(v)) times the FP32 reciprocal of the sum.
 * pred: float[n]; pr: float[n]. Takes 8 bytes of stream-ordered scratch from
 * the library's pool. Does not synchronise. */
int pcpm_ws_init_ranks(const float* pred, uint32_t n, float* pr, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PCPM_WARMSTART_H */
