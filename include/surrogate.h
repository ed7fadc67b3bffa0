/*
 * surrogate.h -- C ABI of the learned surrogate in libinkjet.so.
 *
 * The paper has no learned part.  The surrogate is an added service around
 * the lattice Boltzmann model of inkjet.h: an ensemble of multilayer
 * perceptrons that maps the seven inputs of one ejection run to four
 * outcomes of that run, trained on runs of the lattice Boltzmann model
 * itself, with an acceptance gate that sends every query it cannot answer
 * reliably back to the lattice Boltzmann model.
 *
 *   inputs  x[7]: contact angle (deg), surface tension sigma, drive
 *                 amplitude F0, durations T1, T2, idle time T_idle, nozzle
 *                 width (lattice units)
 *   outcomes y[4]: breakup time (steps), droplet velocity, droplet volume,
 *                 satellite count -- read from the ij_obs records of the run
 *                 (inkjet.h) over the 100 steps after breakup
 *
 * Network (each ensemble member): 7 -> 4 hidden layers of `hidden` units
 * with GELU -> 4, mean-squared error on transformed outcomes, Adam.  Inputs
 * and outcomes are z-scored after an optional log (bit masks below).  Every
 * contraction runs on the 5th-generation tensor cores with BF16 operands and
 * FP32 accumulation (tcgen05.mma, accumulator in tensor memory); master
 * weights, Adam moments and biases are FP32.  Stored operands -- inputs,
 * weights, hidden activations, back-propagated errors -- are BF16.
 *
 * Conventions: as in inkjet.h (every call returns an ij_status; device
 * memory through the allocator callbacks; work on the stream given at
 * creation; calls that return results to the host synchronise it).
 * IJ_ERR_TIMEOUT reports a tensor-core completion wait that ran out of its
 * iteration limit (the kernel then skips its output and returns);
 * IJ_ERR_NUMERIC a non-finite training loss.
 */
#ifndef SURROGATE_H
#define SURROGATE_H

#include "inkjet.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_handle_s* sg_handle;

typedef struct {
  int members;             /* ensemble size, 1..8 */
  int hidden;              /* width of each hidden layer: multiple of 16, 16..256 */
  int batch;               /* training minibatch rows: multiple of 16, 16..65536 */
  float lr, beta1, beta2, eps;   /* Adam */
  unsigned long long seed; /* weight initialisation and minibatch sampling */
  int log_inputs;          /* bit d set: input d is log-transformed before z-scoring */
  int log_outputs;         /* bit d set: outcome d likewise */
  float out_weight[4];     /* loss weight of each outcome */
  int lr_cosine;           /* 1: within each sg_train call lr decays from lr to 0 along a
                              half cosine, lr (1 + cos(pi s / S)) / 2 at step s of S;
                              0: constant lr */
} sg_config;

/* sg_create -- allocate an ensemble and initialise it: He-uniform weights
 * (bound sqrt(6 / fan_in)) from SplitMix64 of (seed, member, index), zero
 * biases.  Errors: IJ_ERR_PARAM (config out of range), IJ_ERR_OOM, IJ_ERR_CUDA. */
ij_status sg_create(const sg_config* cfg, ij_alloc_fn alloc, ij_free_fn free_fn, void* ctx,
                    void* stream, sg_handle* out);

/* sg_set_data -- training set: host arrays x [n][7] and y [n][4] (raw units,
 * positive where a log is taken).  Fixes the transforms (mean and standard
 * deviation of each transformed column), the input box [min, max] of each
 * input and the nearest-neighbour cut of the gate (twice the 95th percentile
 * of the leave-one-out nearest-neighbour distances in transformed input
 * space).  n >= 2. */
ij_status sg_set_data(sg_handle h, const float* x, const float* y, int n);

/* sg_train -- `steps` Adam steps of every member, each on its own minibatch
 * of `batch` rows drawn with replacement (lr constant, or decaying over these
 * steps with lr_cosine).  *loss (may be NULL) receives the
 * mean over members of the last step's loss.  Synchronises. */
ij_status sg_train(sg_handle h, int steps, double* loss);

/* sg_predict -- outcomes of n queries x [n][7]: the ensemble mean [n][4]
 * and standard deviation over members [n][4] in raw units, and (accept may
 * be NULL) the gate: accept[i] = 1 when query i lies in the training input
 * box, within the nearest-neighbour cut of a training point, and the
 * ensemble's standard deviation of breakup time (of droplet velocity) is
 * below tau (tau_v) times the mean's magnitude; else 0 (re-run on the
 * lattice Boltzmann model).  Buffers are device pointers if on_device, else host. */
ij_status sg_predict(sg_handle h, const float* x, int n, float* mean, float* sd, int* accept,
                     int on_device);

/* sg_set_gate -- the relative ensemble spread allowed on breakup time
 * (tau) and on droplet velocity (tau_v), and the nearest-neighbour cut
 * (nn_cut <= 0 keeps the one sg_set_data chose).  Defaults: 0.01, 0.01. */
ij_status sg_set_gate(sg_handle h, float tau, float tau_v, float nn_cut);

/* sg_param_count -- FP32 parameters per member.  Layout of one member: for
 * layers l = 0..4, Wt_l [out][in] then b_l [out], with in = (16, H, H, H, H)
 * and out = (H, H, H, H, 16); input columns 7..15 and output rows 4..15 are
 * padding and stay zero. */
ij_status sg_param_count(sg_handle h, long long* count);
ij_status sg_get_params(sg_handle h, int member, float* out);
ij_status sg_set_params(sg_handle h, int member, const float* in);

/* sg_get_transform -- the transforms fixed by sg_set_data: mean and scale
 * of the 7 inputs and of the 4 outcomes (after the log where selected). */
ij_status sg_get_transform(sg_handle h, float* in_mean, float* in_scale, float* out_mean,
                           float* out_scale);

/* sg_gradients -- one forward and backward pass of every member on the
 * given n rows (x [n][7], y [n][4] raw; n a multiple of 16, <= batch)
 * without an update: grads [members][param_count] (host) and the loss of
 * each member [members] (host, may be NULL). */
ij_status sg_gradients(sg_handle h, const float* x, const float* y, int n, float* grads,
                       double* loss);

ij_status sg_destroy(sg_handle h);
const char* sg_last_error(void);

/* sg_gemm_bf16 -- the tensor-core contraction alone: C [M][N] (FP32, ldc) =
 * A [M][K] (BF16, lda) times B [N][K]^T (BF16, ldb), device pointers, on
 * `stream`.  K, lda, ldb multiples of 8; pointers 16-byte aligned.
 * Synchronises and returns IJ_ERR_TIMEOUT as above. */
ij_status sg_gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K,
                       float* C, int ldc, void* stream);

#ifdef __cplusplus
}
#endif
#endif
