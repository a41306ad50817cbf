/*
 * spnn.h -- C ABI of libspnn, the learned fluence surrogate: a 3D U-Net
 * that maps a voxel pore mask and the solid optics (mu_s h, mu_a h, g) to
 * the log of the voxel fluence Phi/S0 that the Monte Carlo engine (spmc.h)
 * tallies (arXiv 2604.13929, Sec. 2.6 estimators), for screening mask
 * designs (Sec. 5) faster than a photon run.  The paper defines no network;
 * the layers are plain convolutions:
 *
 *   conv3  3x3x3, stride 1, zero padding 1; taps t = (dz, dy, dx) in
 *          {-1,0,1}^3, index (dz+1)*9 + (dy+1)*3 + (dx+1)
 *   down   2x2x2, stride 2; taps o = (oz, oy, ox) in {0,1}^3, index oz*4+oy*2+ox
 *   up     transposed 2x2x2, stride 2: y[2v + o] = b + x[v] W[o]
 *
 * Layout: activations are BF16 in "chunk planes" [C/8][B][D][H][W][8]: each
 * plane holds 8 channels of every voxel (16 bytes per voxel, x fastest), so
 * runs of voxels are contiguous for the TMA loads.  Every channel count is
 * a multiple of 16 and every spatial extent a power of two.  Master weights are FP32 W[taps][cin][cout]; the kernels
 * read them through BF16 "packed" copies made by spnn_pack_weights.
 * Arithmetic: BF16 operands, FP32 accumulation on the tensor cores
 * (tcgen05, accumulators in TMEM), BF16 layer outputs, FP32 weight
 * gradients.
 *
 * Pointers: every tensor argument is a DEVICE pointer owned by the caller
 * unless stated; "stream" is a cudaStream_t (NULL = legacy default stream).
 * All calls are asynchronous and stream-ordered.  Return value: 0
 * (SPNN_OK) or a negative SPNN_E* code; spnn_last_error() gives a
 * thread-local message.  There is no CPU path: without a GPU every call
 * returns SPNN_ECUDA.
 *
 * Concurrency: a forward or input-gradient GEMM (spnn_layer_forward,
 * spnn_layer_dgrad and the network calls built on them) zeroes one of 64
 * device tile counters on its stream before its launch, taken in turn; calls
 * may run concurrently on different streams as long as fewer than 64 of them
 * are in flight at once.
 */
#ifndef SPNN_H
#define SPNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPNN_OK 0
#define SPNN_EINVAL (-1)   /* bad sizes, channel counts or null pointers        */
#define SPNN_ENOMEM (-2)   /* device allocation failed                          */
#define SPNN_ECUDA (-3)    /* CUDA error, no device, or a kernel wait timed out */

#define SPNN_CONV3 0
#define SPNN_DOWN 1
#define SPNN_UP 2

#define SPNN_PACK_FWD 0    /* operand of spnn_layer_forward                     */
#define SPNN_PACK_DGRAD 1  /* operand of spnn_layer_dgrad                       */

const char* spnn_last_error(void);
int spnn_version(void);
/*
 * Synchronise the stream and report kernel-side failures: SPNN_ECUDA if a
 * CUDA error is pending or a kernel gave up on a bounded wait since the last
 * call (the flag is then cleared), else SPNN_OK.
 */
int spnn_status(void* stream);

/*
 * Launch tuning of the GEMM kernels, process-wide (0 = automatic):
 *   SPNN_OPT_CONV_SUBTILES  128-row subtiles per CTA of a conv3 GEMM (1, 2, 4),
 *                           stacked along y, sharing one halo box and weight copy
 *   SPNN_OPT_CONV_PLANES    8-channel chunk planes per conv3 K-step (2, 4)
 *   SPNN_OPT_STAGE_KB       shared-memory budget of the stage ring in KB (<= 220)
 *   SPNN_OPT_WGRAD_HALO     1 (default): conv3 weight gradients with at most 32
 *                           output channels on halo K-steps (one input box and
 *                           three shifted output-gradient boxes per x-run);
 *                           2: wherever they fit (up to 80 output channels);
 *                           0: always the per-tap kernel
 *   SPNN_OPT_CONV_FULL_HALO 1: conv3 forward / input gradient on 8 x 16 tiles whose
 *                           one box per plane block serves all 27 taps, where it
 *                           fits; 0 (default): one box per x-shift
 *   SPNN_OPT_ROWS_PERSISTENT k in 1..16: forward / input-gradient GEMMs launch k
 *                           CTAs per resident slot that the occupancy query
 *                           reports (default 2: the query has answered one CTA
 *                           per SM where two are resident), each claiming tiles
 *                           in order until none are left; 0: one CTA per tile
 *   SPNN_OPT_LOSS_FLUENCE_WEIGHT 1: spnn_unet_backward weighs each voxel's
 *                           squared error by exp(target) over its sample's mean
 *                           of exp(target) (targets are log fluences); 0
 *                           (default): unweighted
 * Settings that do not fit a layer fall back to the automatic choice.
 */
#define SPNN_OPT_CONV_SUBTILES 1
#define SPNN_OPT_CONV_PLANES 2
#define SPNN_OPT_STAGE_KB 3
#define SPNN_OPT_WGRAD_HALO 4
#define SPNN_OPT_CONV_FULL_HALO 5
#define SPNN_OPT_ROWS_PERSISTENT 7
#define SPNN_OPT_LOSS_FLUENCE_WEIGHT 8
int spnn_set_option(int key, int value);

/* Elements (BF16) of a packed weight operand for a layer. */
size_t spnn_packed_elems(int kind, int cin, int cout);
/* FP32 w[taps][cin][cout] (device) -> packed BF16 operand (device, spnn_packed_elems). */
int spnn_pack_weights(int kind, int cin, int cout, int which, const float* w, void* packed, void* stream);

/*
 * One layer forward: y = act(layer([x0, x1]) + bias).
 *   B, D, H, W   grid of the layer INPUT (D, H, W powers of two; the row
 *                grid -- output grid for conv3/down, input grid for up --
 *                must hold a multiple of 128 voxels).
 *   x0 (c0 ch), x1 (c1 ch, conv3 only, may be NULL with c1 = 0): inputs,
 *                concatenated along channels, x0 first.
 *   packed       SPNN_PACK_FWD operand;  bias: FP32 [cout] or NULL.
 *   relu         0 / 1.
 *   y            output (B, D', H', W', cout): D' = D (conv3), D/2 (down), 2D (up).
 *   head_w, head_b, head_out: optional fused one-channel head (conv3,
 *                cout <= 256; FP32 device [cout], scalar, [rows]):
 *                head_out[v] = *head_b + sum_c y[v, c] head_w[c] in FP32 from
 *                the BF16-rounded y.  NULL to skip.
 */
int spnn_layer_forward(int kind, int B, int D, int H, int W, const void* x0, int c0, const void* x1, int c1,
                       const void* packed, const float* bias, int cout, int relu, void* y,
                       const float* head_w, const float* head_b, float* head_out, void* stream);

/*
 * Input gradient of one layer.  dy: gradient w.r.t. the layer's
 * pre-activation output (cout channels, output grid).  Writes
 *   dx0[v, c] = (g[v, c] + addend0[v, c]) * (mask0[v, c] > 0)   for c < c0
 *   dx1[v, c - c0] likewise with addend1 / mask1                 for c >= c0
 * where g is the adjoint of the layer applied to dy; addends and masks are
 * optional (NULL), dx1 only for a concatenated conv3 input.  B, D, H, W:
 * grid of the layer INPUT.  packed: SPNN_PACK_DGRAD operand.
 */
int spnn_layer_dgrad(int kind, int B, int D, int H, int W, const void* dy, int cout, const void* packed,
                     int c0, int c1, void* dx0, const void* addend0, const void* mask0, void* dx1,
                     const void* addend1, const void* mask1, void* stream);

/*
 * Weight and bias gradients of one layer, ADDED (FP32 atomics) into
 * dw[taps][c0 + c1][cout] and db[cout] (db may be NULL).  x0, x1 as in
 * spnn_layer_forward; dy as in spnn_layer_dgrad.
 */
int spnn_layer_wgrad(int kind, int B, int D, int H, int W, const void* x0, int c0, const void* x1, int c1,
                     const void* dy, int cout, float* dw, float* db, void* stream);

/* ---------------------------------------------------------------- data -- */

/*
 * Input features, BF16 chunk planes [2][B][D][H][W][8] (16 channels):
 * 0 pore (mask == 1), 1 solid, 2 ln(mu_s h), 3 ln(mu_a h)/4, 4 g,
 * 5 (z + 1/2)/D, 6 -mu_eff (z + 1/2)/8, 7 porosity phi, 8..15 zero, where phi
 * is the sample's pore fraction and mu_eff = sqrt(3 mu_a' (mu_a' + mu_s'(1-g)))
 * the diffusion attenuation (Sec. 2.4) of the medium scaled to its solid
 * fraction, mu' = (1 - phi) mu (Eq. EMA_scaling).  Uses a B-float scratch
 * from the stream-ordered allocator.
 * mask: uint8 (B, D, H, W), 1 = pore;  optics: FP32 (B, 3) = (mu_s h, mu_a h, g).
 */
int spnn_pack_input(const uint8_t* mask, const float* optics, int B, int D, int H, int W, void* x, void* stream);

/*
 * Training target: out[v] = ln max(F[v] * W * H / (N_b * 2^32), floor) from
 * the Monte Carlo's Q32.32 track-length field F (uint64, (B, D, H, W), x
 * fastest); n_photons: FP64 [B] photons of each sample (Sec. 2.6 steady-state
 * normalisation Phi/S0 = F nx ny / N).
 */
int spnn_log_fluence(const uint64_t* raw, const double* n_photons, int B, int D, int H, int W, float floor_,
                     float* out, void* stream);

/*
 * Per-phase depth profiles of Phi = exp(log_phi): prof[b][0][z] mean over
 * the solid voxels of layer z, prof[b][1][z] over the pores (NaN where a
 * layer has none).  log_phi FP32 (B, D, H, W), mask uint8, prof FP32 (B, 2, D).
 */
int spnn_phase_profiles(const float* log_phi, const uint8_t* mask, int B, int D, int H, int W, float* prof,
                        void* stream);

/* ------------------------------------------------------------- network -- */

/*
 * The U-Net: base width c0 (16 or 32; widths c0, 2c0, 4c0, 8c0), cubes of
 * edge n (power of two, n >= 16; batch * (n/8)^3 a multiple of 128), up to
 * max_batch samples.
 * Layers in order e0a e0b d1 e1a e1b d2 e2a e2b d3 b1 b2 u2 c2a c2b u1 c1a
 * c1b u0 c0a c0b + head; decoder "a" layers read [up, skip].  Parameters are
 * one flat FP32 vector: per layer W[taps][cin][cout] then b[cout], then the
 * head's w[c0] and b.  Owns all device buffers (activations of max_batch
 * samples, gradients, Adam moments).  Returns NULL on error.
 */
typedef struct spnn_unet spnn_unet_t;
spnn_unet_t* spnn_unet_create(int c0, int n, int max_batch);
void spnn_unet_destroy(spnn_unet_t* net);
size_t spnn_unet_param_count(const spnn_unet_t* net);
/* params: host FP32 [param_count].  set also repacks the BF16 operands. */
int spnn_unet_set_params(spnn_unet_t* net, const float* params);
int spnn_unet_get_params(spnn_unet_t* net, float* params);
/* grads: host FP32 [param_count], from the last spnn_unet_backward. */
int spnn_unet_get_grads(spnn_unet_t* net, float* grads);
/* Forward of `batch` samples: x BF16 chunk planes [2][batch][n][n][n][8]; pred FP32 (batch, n^3). */
int spnn_unet_forward(spnn_unet_t* net, const void* x, int batch, float* pred, void* stream);
/*
 * Backward of the last forward (same x, same batch): loss = mean w (pred -
 * target)^2 over batch * n^3 voxels (w = 1, or the fluence weights of
 * SPNN_OPT_LOSS_FLUENCE_WEIGHT), accumulated into *loss (FP64 device
 * scalar, caller zeroes it; may be NULL); gradients overwrite the
 * network's gradient buffer.
 */
int spnn_unet_backward(spnn_unet_t* net, const float* target, int batch, double* loss, void* stream);
/* One Adam step (Kingma and Ba 2015) on the gradient buffer, then repack. */
int spnn_unet_adam(spnn_unet_t* net, float lr, float beta1, float beta2, float eps, void* stream);
/*
 * Copy the BF16 output of a layer (index in the order above) of the last
 * forward's `batch` samples into dst (device, chunk planes [cout/8][batch][e][e][e][8]).
 */
int spnn_unet_copy_activation(spnn_unet_t* net, int layer, int batch, void* dst, void* stream);
/* Shape of a layer's output: edge e and channels. */
int spnn_unet_layer_shape(const spnn_unet_t* net, int layer, int* edge, int* channels);

#ifdef __cplusplus
}
#endif
#endif
