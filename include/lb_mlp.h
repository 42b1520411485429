/*
 * lb_mlp.h -- C ABI of the learned surrogate for the filling curve l(t).
 *
 * The paper has no surrogate: it measures l(t) from lattice Boltzmann runs and
 * compares with Washburn's law (Eqs. 1-3).  This library learns the map from a
 * capillary's parameters to its filling curve from runs of the batched lattice
 * Boltzmann sweep (lb_batch_run_sampled), so that a sweep over parameters can
 * be answered without running the LB, and falls back to the LB (the reference
 * for its error) wherever its ensemble disagrees.
 *
 * Network (per ensemble member): x (n_in) -> tanh(W1 x + b1) (n_hidden) ->
 * tanh(W2 h1 + b2) (n_hidden) -> W3 h2 + b3 (n_out).  The contractions run on
 * tensor cores with BF16 operands (weights and activations) and FP32
 * accumulation; FP32 master weights are updated by AdamW.  All members are
 * trained and evaluated in the same launches.
 *
 * Parameter layout (one member, FP32, flattened): W1 [n_hidden][n_in], b1
 * [n_hidden], W2 [n_hidden][n_hidden], b2 [n_hidden], W3 [n_out][n_hidden],
 * b3 [n_out].  Data arrays are row-major [batch][n_in] / [batch][n_out] FP32.
 * Every function returns lb_status (values of include/lb.h) and issues its work
 * on the stream given to lb_mlp_create; calls that return host data wait.
 */
#ifndef LB_MLP_GB300_H
#define LB_MLP_GB300_H

#include "lb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_mlp lb_mlp;

/* Create members with Glorot-uniform weights from a counter-based generator
 * seeded by seed (member m uses seed + m), zero biases.  n_in <= 16,
 * n_hidden % 64 == 0 and <= 1024, n_out % 8 == 0 and <= 1024, 1 <= members
 * <= 16, 1 <= max_batch <= 4194240 (65535 row tiles of 64), else
 * LB_ERR_ARG.  Device memory through alloc (may be NULL). */
lb_status lb_mlp_create(int n_in, int n_hidden, int n_out, int members, int max_batch,
                        unsigned long long seed, const lb_alloc *alloc, void *stream, lb_mlp **out);
void lb_mlp_destroy(lb_mlp *m);

/* Number of FP32 parameters of one member. */
long lb_mlp_num_params(const lb_mlp *m);

/* Read or replace the FP32 master parameters of member k (host arrays of
 * lb_mlp_num_params floats); set also refreshes the BF16 working copy and
 * clears that member's AdamW moments. */
lb_status lb_mlp_get_params(lb_mlp *m, int k, float *params);
lb_status lb_mlp_set_params(lb_mlp *m, int k, const float *params);

/* Load a training set of n rows (host arrays), kept on the device. */
lb_status lb_mlp_set_data(lb_mlp *m, int n, const float *x, const float *y);

/* Gradients of the mean squared error (1/(n n_out)) sum (f(x) - y)^2 of member
 * k on the loaded data with respect to its parameters (host array of
 * lb_mlp_num_params floats, same layout).  No update is made. */
lb_status lb_mlp_gradients(lb_mlp *m, int k, float *grads, float *loss);

/* steps AdamW updates of every member on the loaded data (full batch): lr,
 * betas (0.9, 0.999), eps 1e-8, decoupled weight decay wd on the weights (not
 * the biases).  The learning rate follows a cosine from lr down to lr_min over
 * the steps.  losses (host, may be NULL) receives each member's final loss. */
lb_status lb_mlp_train(lb_mlp *m, int steps, float lr, float lr_min, float wd, float *losses);

/* Forward pass of every member on n rows of x (host): mean and standard
 * deviation over members of each output (host [n][n_out]); members (may be
 * NULL) receives every member's output [k][n][n_out]. */
lb_status lb_mlp_predict(lb_mlp *m, int n, const float *x, float *mean, float *stddev, float *members);

const char *lb_mlp_last_error(const lb_mlp *m);

#ifdef __cplusplus
}
#endif

#endif /* LB_MLP_GB300_H */
