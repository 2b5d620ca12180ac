/*
 * paradeisos_mlp.h -- learned Lanczos start vector (C ABI).
 *
 * Not part of the paper (arXiv 1707.03974): an addition that trains a small
 * network on ground states computed by the library itself and uses it to build
 * start vectors for lanczos_ground_state.  The network maps the n_in = 2L
 * occupation bits of a combined basis state (bit i of (up << L) | dn, the
 * layout of Sec. III) to (log|psi|, sign logit):
 *     z1 = W1 x + b1, a1 = gelu(z1), z2 = W2 a1 + b2, a2 = gelu(z2), out = W3 a2 + b3,
 * hidden width 128, gelu the tanh form x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715
 * x^3))) (Hendrycks & Gimpel 2016), tanh by the hardware's tanh.approx.f32
 * (relative error about 2^-11, below the bfloat16 rounding of the
 * activations).  Parameters are one float32
 * vector in the order W1 [128 x n_in] row-major, b1 [128], W2 [128 x 128],
 * b2 [128], W3 [2 x 128], b3 [2]; matrix products run on the tensor cores
 * (tcgen05, bfloat16 operands, float32 accumulation).  All pointers are device
 * memory unless stated; calls are asynchronous on `stream` unless stated.
 */
#ifndef PARADEISOS_MLP_H
#define PARADEISOS_MLP_H

#include "paradeisos.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hb_mlp *hb_mlp_handle;

/* New network for n_in (1..32) input bits; weights uniform(+-1/sqrt(fan_in))
 * from SplitMix64(seed), biases zero.  Synchronous. */
hb_status mlp_create(int n_in, uint64_t seed, hb_mlp_handle *out);
hb_status mlp_destroy(hb_mlp_handle m);
hb_status mlp_param_count(hb_mlp_handle m, uint64_t *P);
/* HOST float arrays of mlp_param_count elements; synchronous. */
hb_status mlp_get_params(hb_mlp_handle m, float *host_params);
hb_status mlp_set_params(hb_mlp_handle m, const float *host_params);
/* out[n][2] = (log|psi|, sign logit) of combined states (uint64). */
hb_status mlp_forward(hb_mlp_handle m, const uint64_t *states, uint64_t n, float *out, void *stream);
/* Loss  sum_r w_r [ (out0_r - t_log_r)^2 + lam softplus(-t_sign_r out1_r) ]  (w normalised by
 * the caller) and its gradient w.r.t. the parameters, kept in the handle for
 * mlp_adam_step; grad (device float[P]) and loss (device float) may be NULL. */
hb_status mlp_gradient(hb_mlp_handle m, const uint64_t *states, uint64_t n, const float *t_log,
                       const float *t_sign, const float *weights, float lam, float *grad, float *loss,
                       void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the last gradient. */
hb_status mlp_adam_step(hb_mlp_handle m, float lr, void *stream);
/* Start vector over the whole basis of h (n_in must be 2L): v[I] = sign * exp(min(log|psi|, 10) - 10)
 * for every combined index I (states from the backward map), in dtype dt.  Not normalised. */
hb_status mlp_start_vector(hb_mlp_handle m, hb_handle h, hb_dtype dt, void *v, void *stream);
/* Training samples for the network: n basis states of h drawn with probability psi_I^2 / sum psi^2
 * (inverse-CDF sampling over the whole basis; draw i is SplitMix64 output i + 1 of the stream seeded
 * with `seed`, mapped to [0, 1)), written as combined strings (states, uint64 [n]) with the targets
 * t_log = log|psi_I| minus its mean over the n draws and t_sign = +-1, after the global sign of psi
 * is fixed so that its entry of largest magnitude (lowest index on ties) is positive.  psi: device
 * float[D] (need not be normalised).  workspace: device buffer of mlp_sample_workspace_bytes bytes,
 * 256-byte aligned.  Real-space handles only.  Asynchronous on `stream`. */
hb_status mlp_sample_workspace_bytes(hb_handle h, uint64_t n, uint64_t *bytes);
hb_status mlp_sample_training(hb_handle h, const float *psi, uint64_t n, uint64_t seed, uint64_t *states, float *t_log,
                              float *t_sign, void *workspace, uint64_t workspace_bytes, void *stream);
/* Sticky device error (HB_ERR_TIMEOUT if a tensor-core completion wait gave up); synchronises. */
hb_status mlp_last_error(hb_mlp_handle m);
/* Test entry: C[M x N] = A[M x K] B[N x K]^T, A and B bfloat16 row-major, C float32 row-major,
 * computed by the library's tcgen05 kernel (K multiple of 8, N = 32 or a multiple of 128).
 * Synchronises `stream`. */
hb_status mlp_tc_gemm(const void *A, const void *B, float *C, int M, int N, int K, void *stream);

/* Test entry: y[i] = gelu(x[i]) (deriv 0) or gelu'(x[i]) (deriv 1), the activation exactly as the
 * network's kernels evaluate it (the tanh form above; the derivative is that form's exact
 * derivative).  Asynchronous. */
hb_status mlp_activation(const float *x, uint64_t n, float *y, int32_t deriv, void *stream);

/* Failure-detection self test (synchronous): a kernel waits, with the bounded
 * mbarrier wait used by the tensor-core kernels, on a barrier that nothing
 * arrives at; returns HB_ERR_TIMEOUT after max_tries polls (the device stays
 * usable), HB_OK never (nothing arrives), HB_ERR_CUDA on a runtime error. */
hb_status hb_device_wait_selftest(uint32_t max_tries);

#ifdef __cplusplus
}
#endif
#endif /* PARADEISOS_MLP_H */
