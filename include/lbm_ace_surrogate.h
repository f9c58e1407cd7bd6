/*
 * lbm_ace_surrogate.h -- C ABI of the learned surrogate for the phase field of the
 * lattice Boltzmann interface-capturing scheme (H. Liang, arXiv 2203.05230).
 *
 * The paper has no learned component; this is an accelerator built around its
 * method. One application of the network advances phi by K = 16 lattice Boltzmann
 * steps of the scheme of Eqs. 9-13 under a prescribed velocity:
 *
 *     x0  = (phi, 20 u, 20 v)                                  3 input channels
 *     z_l = conv3x3(a_{l-1}, W_l) + b_l,  a_l = GELU(z_l)      l = 1..4, 32 channels
 *     z_5 = conv3x3(a_4, W_5) + b_5                            1 channel
 *     phi_out = phi + z_5 - mean(z_5)                          mean over each image
 *
 * conv3x3 is the periodic 3x3 cross-correlation (out[co][y][x] = b[co] +
 * sum W[co][ci][j][i] in[ci][y+j-1][x+i-1], indices modulo the image), GELU(z) =
 * z Phi(z) with Phi the standard normal CDF. Removing the mean of z_5 conserves
 * sum(phi), the global mass that Eq. 8's divergence form conserves.
 *
 * Arithmetic: layers 2-5 (97 % of the multiply-adds) and the input gradients of
 * layers 2-4 run on the fifth-generation tensor cores (tcgen05.mma, BF16 weights and
 * activations, FP32 accumulation in tensor memory); the weight gradients of layers
 * 2-4 on the tensor cores through mma.sync; layer 1 (3 input channels) and the layer-5
 * and layer-1 gradients on the FP32 units (layer 1 with FP32 weights). Stored
 * activations z_l, a_l and back-propagated gradients dL/dz_l of layers 1-4 are BF16;
 * phi, u, v, phi_out, z_5, the loss and the weight gradients are FP32 (gradient sums
 * over pixels in FP64 across CTAs).
 *
 * Conventions (as in lbm_ace.h): every function returns a status (LBM_ACE_OK = 0,
 * negative on error, codes of lbm_ace.h) and never aborts; messages through
 * lbm_ace_net_last_error. Image arrays are DEVICE pointers on the net's device to
 * FP32 [batch][ny][nx] (x fastest), owned by the caller, valid until the stream has
 * passed the call. Device work is issued on the stream given at creation; functions
 * that return values to the host synchronise it. The net owns its device memory,
 * which grows on demand to the largest batch * ny * nx seen.
 */
#ifndef LBM_ACE_SURROGATE_H
#define LBM_ACE_SURROGATE_H

#include <stddef.h>

#include "lbm_ace.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ACE_NET_WIDTH 32     /* hidden channels */
#define LBM_ACE_NET_K 16         /* lattice Boltzmann steps per application */
#define LBM_ACE_NET_PARAMS 28929 /* 3->32->32->32->32->1, 3x3 kernels, with biases */

typedef struct lbm_ace_net lbm_ace_net; /* opaque */

/* Create a network on CUDA device `device`, issuing work on `stream` (a
 * cudaStream_t; NULL for the legacy default stream). Parameters start at zero. */
int lbm_ace_net_create(int device, void* stream, lbm_ace_net** out);

/* Parameters as one flat FP32 host vector of LBM_ACE_NET_PARAMS values, in the order
 * W_1, b_1, ..., W_5, b_5, each W in [co][ci][j][i] order (j the row offset, i the
 * column offset, 0..2). set_params resets the Adam moments and step count;
 * count must equal LBM_ACE_NET_PARAMS. Synchronous. */
int lbm_ace_net_set_params(lbm_ace_net* net, const float* params, size_t count);
int lbm_ace_net_get_params(lbm_ace_net* net, float* params, size_t count);

/* phi_out = network(phi, u, v) for `batch` periodic images of ny x nx (each >= 3).
 * phi_out may alias neither input. Asynchronous. */
int lbm_ace_net_forward(lbm_ace_net* net, const float* phi, const float* u, const float* v, float* phi_out,
                        int batch, int ny, int nx);

/* Forward, mean squared error L = mean((phi_out - target)^2) over all batch*ny*nx
 * nodes, and its gradient with respect to the parameters (kept on the device for
 * lbm_ace_net_adam). If loss is not NULL, *loss receives L (synchronous); if grad is
 * not NULL it receives the gradient (count == LBM_ACE_NET_PARAMS, synchronous);
 * with both NULL the call is asynchronous. */
int lbm_ace_net_loss_grad(lbm_ace_net* net, const float* phi, const float* u, const float* v, const float* target,
                          int batch, int ny, int nx, double* loss, float* grad, size_t count);

/* One Adam step (Kingma and Ba, 2015, with bias correction) on the gradient of the
 * last loss_grad: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). Asynchronous. */
int lbm_ace_net_adam(lbm_ace_net* net, float lr, float beta1, float beta2, float eps);

/* dst[k] = src[index[k]] for k < count, where each image has image_elems FP32 values
 * (device pointers; index is a HOST array of image indices, each checked >= 0 only:
 * the caller guarantees they are inside src). Asynchronous device-to-device copies. */
int lbm_ace_net_gather(lbm_ace_net* net, float* dst, const float* src, const long long* index, int count,
                       long long image_elems);

/* Checks of a single phase field phi (device, [ny][nx]): *mass = sum phi (FP64), and
 * *width = sum phi (1 - phi) / sum |grad phi| over the nodes with 0.05 < phi < 0.95
 * (central differences, periodic), which estimates the interface parameter eps of the
 * equilibrium profile phi = 1/2 + 1/2 tanh(s / (2 eps)) (Eq. 2; 0 if no node lies in
 * the band). Either pointer may be NULL. Synchronous. */
int lbm_ace_net_metrics(lbm_ace_net* net, const float* phi, int ny, int nx, double* mass, double* width);

/* Block until the net's device work has finished. */
int lbm_ace_net_synchronize(lbm_ace_net* net);

/* Failure self-test of the tensor-core kernels' bounded waits (a service of this
 * library; the paper has no counterpart). One thread waits, with the same bounded
 * mbarrier wait those kernels use, on a barrier that nothing arrives on, gives up after
 * limit_cycles SM clock cycles (1 .. 2e9, the kernels' own limit) and raises the net's
 * error flag as they would; no tensor-core operation runs and no tensor memory is held.
 * Synchronous. Returns LBM_ACE_ETIMEOUT, the expected result, and clears the flag: the
 * net then works as before. LBM_ACE_EINVAL for a limit out of range. */
int lbm_ace_net_wait_selftest(lbm_ace_net* net, long long limit_cycles);

/* Launch shape of the persistent tensor-core kernels: CTAs launched (at most) for the
 * hidden layers and for layer 5, the resident CTAs per SM the occupancy calculator
 * reports for each, and the SM count. Any pointer may be NULL. */
int lbm_ace_net_launch_shape(const lbm_ace_net* net, int* conv_ctas, int* conv_occupancy, int* out_ctas,
                             int* out_occupancy, int* sms);

const char* lbm_ace_net_last_error(const lbm_ace_net* net);

/* Release all device memory (NULL-safe). */
void lbm_ace_net_destroy(lbm_ace_net* net);

/* ---- Hybrid advance: surrogate windows with a lattice Boltzmann fallback -----------
 * Advances the lattice by `windows` windows of K = 16 steps. Each window applies the
 * network to phi(t) with the velocity u(t + K/2) and accepts the result unless its
 * mass drifts from the mass at the start of the call by more than mass_tol
 * (relative) or its interface width (lbm_ace_net_metrics) deviates from the width at
 * the start by more than width_tol (relative); a rejected window is advanced by K
 * lattice Boltzmann steps instead, restarting the lattice from the current phi
 * (lbm_ace_reset_device) when surrogate windows came before. On return the lattice
 * holds phi at t0 + K * windows (restarted from the surrogate's field if the last
 * window was a surrogate window). The lattice may have any storage precision and a
 * vortex, uniform or field velocity; it must work on the same stream as the net.
 * Up to 8 surrogate windows run back to back on the device before the host reads
 * their checks (one synchronisation per group; the group shrinks to one window after a
 * rejection and doubles after each group without one); the windows after a rejected
 * one are discarded, so the result is the same as checking window by window.
 * stats (may be NULL) receives the counts and the extreme deviations accepted. */
typedef struct {
    long long windows;           /* windows advanced */
    long long surrogate_windows; /* windows advanced by the network */
    long long fallback_windows;  /* windows advanced by K lattice Boltzmann steps */
    double mass0, width0;        /* mass and width at the start of the call */
    double max_mass_drift;       /* largest relative mass drift of an accepted window */
    double max_width_dev;        /* largest relative width deviation of an accepted window */
} lbm_ace_hybrid_stats;

int lbm_ace_hybrid_advance(lbm_ace_ctx* lattice, lbm_ace_net* net, long long windows, double mass_tol,
                           double width_tol, lbm_ace_hybrid_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* LBM_ACE_SURROGATE_H */
