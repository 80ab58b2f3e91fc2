/*
 * fh_nn.h -- C ABI of the learned warm start's network (part of libfh.so).
 *
 * The paper has no network; this is the learned warm-start pattern built on
 * top of the method: a small 3-D convolutional network maps a description of
 * the microstructure to the fluctuation fields e^(b) - e_b of the d unit
 * loads; the caller forms a warm start from it, projects it onto the
 * admissible fields with fh_project_compatible (fh.h), and runs CG from there
 * with the cold start e = E as fallback.
 *
 * Network (all kernels hand-written, float32 activations, bfloat16-rounded
 * weights, float32 accumulation; levels N, N/3, N/9, N/27; channels c0..c3;
 * layers 0..10 in parameter order).  The forward convolutions and the data
 * gradients run on the tensor cores (tcgen05, each float32 activation or
 * gradient split into two bfloat16 halves), the weight gradients on the CUDA
 * cores:
 *   a0 = leaky(conv0(x))            a1 = leaky(conv1(pool(a0)))
 *   a2 = leaky(conv2(pool(a1)))     a3 = leaky(conv3(pool(a2)))
 *   v2 = up(leaky(conv4(a3))) + a2  u2 = leaky(conv5(v2))
 *   v1 = up(leaky(conv6(u2))) + a1  u1 = leaky(conv7(v1))
 *   v0 = up(leaky(conv8(u1))) + a0  u0 = leaky(conv9(v0))
 *   y  = conv10(u0)
 * conv: 3x3x3, periodic padding, bias; pool: mean over 3x3x3 blocks; up:
 * nearest-neighbour upsampling by 3; leaky: max(x,0) + 0.1 min(x,0).
 * Parameters are one flat float32 vector: for each of the 11 layers in order,
 * its weights [out][in][27] (taps ordered dz, dy, dx in {-1,0,1}, dx fastest)
 * then its biases [out].
 * Fields are [channels][N0][N1][N2] float32 device arrays.
 */
#ifndef FH_NN_H_
#define FH_NN_H_

#include "fh.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fh_nn fh_nn;

/* Create a network for grids N (3 ints, each a multiple of 27), cin input and
 * cout output channels (each <= 64), channels[4] = (c0, c1, c2, c3), each
 * <= 64, or NULL for (16, 32, 48, 64).  Parameters start at zero (set them
 * with fh_nn_set_params).  stream: cudaStream_t or NULL.
 * Errors: FH_ERR_ARG, FH_ERR_OOM, FH_ERR_CUDA (FH_ERR_TIMEOUT from the
 * synchronising calls if a tensor-core kernel's bounded wait expired). */
fh_status fh_nn_create(fh_nn** out, const int* N, int cin, int cout, const int* channels, void* stream);

/* Number of float32 parameters. */
long long fh_nn_param_count(const fh_nn* nn);

/* Kernels launched by this network so far. */
long long fh_nn_launches(const fh_nn* nn);

/* Copy parameters in (host, count floats; also resets the Adam moments) or out. */
fh_status fh_nn_set_params(fh_nn* nn, const float* host, long long count);
fh_status fh_nn_get_params(fh_nn* nn, float* host, long long count);

/* y = net(x); x: device [cin][N...], y: device [cout][N...].  Asynchronous. */
fh_status fh_nn_forward(fh_nn* nn, const float* x, float* y);

/* Forward, mean-squared-error loss against target (device [cout][N...]) and
 * backward.  *loss (host, may be NULL) receives the loss; grad_host (host,
 * param_count floats, may be NULL) receives the gradient.  Synchronises. */
fh_status fh_nn_gradients(fh_nn* nn, const float* x, const float* target, double* loss, float* grad_host);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias correction with the
 * 1-based step count) on the gradients of the MSE loss at (x, target). */
fh_status fh_nn_train_step(fh_nn* nn, const float* x, const float* target, float lr, int step, double* loss);

void fh_nn_destroy(fh_nn* nn);

/* Network input from a phase image (device, nodes bytes) and its isotropic
 * phase table L (host, nphase*d*d float64): channel 0 = log10(L_p / L_0) / 4,
 * channel 1 = 1 for inclusions (p > 0).  x: device float32 [2][nodes].
 * Synchronises.  Errors: FH_ERR_ARG, FH_ERR_NOT_SPD, FH_ERR_OOM, FH_ERR_CUDA. */
fh_status fh_nn_features(const uint8_t* phase, int nphase, const double* L, int d, long long nodes,
                         float* x, void* stream);

/* First-order response of the cell: x[b*d + a] = (B e_b)_a for the d unit
 * loads e_b, B = F^-1 Gamma0 F dL of Eq. (mtrx_B), i.e. the fluctuation of
 * the first fixed-point iterate of Eq. (orig_fft) started at e = e_b (up to
 * sign).  d products of ctx (float32 where ctx has that pipeline, else
 * float64).  x: device float32 [d*d][nodes] (nodes = product of ctx's N).
 * Synchronises the device.  Errors: FH_ERR_ARG, FH_ERR_OOM, FH_ERR_CUDA. */
fh_status fh_nn_response_features(fh_ctx* ctx, int d, long long nodes, float* x);

/* Training target from the d solved unit-load fields (host array of d device
 * float64 pointers, each [d][nodes]): target[b*d + a] = e^(b)_a - delta_ab
 * + base[b*d + a], device float32 [d*d][nodes].  base (device float32
 * [d*d][nodes], or NULL for zero) is what the network's output is measured
 * from; with base = fh_nn_response_features the network learns the
 * correction to the first-order response.  Asynchronous. */
fh_status fh_nn_targets(const double* const* fields, int d, long long nodes, const float* base, float* target,
                        void* stream);

/* Warm start for load E (host, d float64) from a prediction pred (device
 * float32 [d*d][nodes], as fh_nn_forward returns) and the same base as the
 * targets (or NULL): x0 = E + Q(sum_b E_b (pred_b - base_b)) with Q the
 * compatible projection of ctx (fh_project_compatible), so x0 - E is a
 * zero-mean compatible field.  x0: device float64 [d][nodes].  Synchronises
 * the device. */
fh_status fh_nn_warm_start(fh_ctx* ctx, const float* pred, const float* base, const double* E, int d,
                           long long nodes, double* x0, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FH_NN_H_ */
