/*
 * mm_fno.h - C ABI of the learned relaxation warm start and of the library's
 * tensor-core matrix product.
 *
 * The paper relaxes a start state with the plain solver (Sec. 4: every
 * standard problem starts from a relaxed state; Sec. 6: the scripted
 * relax()).  The warm start predicts a relaxed state of a 128 x 128 x 1 film
 * from its material and applied field with a Fourier neural operator
 * (Li et al., ICLR 2021); mm_relax then finishes the relaxation from that
 * prediction, and the solver's own torque bound judges it.  The operator:
 * lift 16 -> 32 channels, four Fourier layers (16 modes per axis and sign,
 * complex 32 x 32 mixing per mode, point-wise 32 x 32 map, gelu between
 * layers), projection 32 -> 128 (gelu) -> 3.  All products run on the tensor
 * cores with bf16 operands and fp32 accumulation; the truncated transforms
 * use a two-term (hi + lo) bf16 DFT basis.
 *
 * Conventions as in mm.h: device pointers, caller-allocated workspace, work
 * issued asynchronously on the given stream, MM_* status codes
 * (mm_status in mm.h), last error text per context.
 */
#ifndef MM_FNO_H
#define MM_FNO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mm_fno mm_fno;

/* Context for batches of up to max_batch films (a multiple of 8, 8..1024). */
int mm_fno_create(mm_fno** out, int max_batch, void* cuda_stream);

/* Device workspace bytes (weights, Adam moments, DFT bases ~128 MB,
 * activations of max_batch films). */
size_t mm_fno_workspace_bytes(const mm_fno* f);

/* Hand over the workspace (256-byte aligned); clears it and builds the DFT bases. */
int mm_fno_set_workspace(mm_fno* f, void* dev_ptr, size_t bytes);

/*
 * Number of floats of the flat parameter vector, laid out as
 *   lift_w [32][16], lift_b [32],
 *   spectral [4 layers][2: re, im][512 modes][32 out][32 in]
 *     (mode = kx*32 + j, kx = 0..15, ky = j for j < 16, 112 + (j - 16) otherwise),
 *   pw_w [4][32 out][32 in], pw_b [4][32],
 *   proj1_w [128][32], proj1_b [128], proj2_w [3][128], proj2_b [3].
 */
size_t mm_fno_param_count(void);

/* Load the fp32 parameters (device, mm_fno_param_count floats); resets the
 * optimiser's moments and step count.  Needed before training or prediction. */
int mm_fno_set_params(mm_fno* f, const float* params_dev);
/* Copy the current fp32 parameters out (device). */
int mm_fno_get_params(mm_fno* f, float* params_dev);

/*
 * One training step on a batch (a multiple of 8, <= max_batch):
 *   x       device fp32 [batch][16][128][128] input fields
 *   target  device fp32 [batch][3][128][128] relaxed magnetisation
 * forward, loss = mean (out - target)^2, backward, then (lr != 0) one Adam
 * step (beta1, beta2, eps) on the fp32 parameters.  loss_host (may be NULL;
 * non-NULL synchronises) receives the loss before the update; grad_out (device,
 * may be NULL) receives the flat gradient.  MM_ETIMEOUT (with loss_host) if a
 * tensor-core product gave up waiting for its operands.
 */
int mm_fno_train_step(mm_fno* f, const float* x, const float* target, int batch, float lr, float beta1, float beta2,
                      float eps, double* loss_host, float* grad_out);

/* Prediction: m_out (device fp32 [batch][3][128][128], may be NULL) receives
 * the normalised output, raw_out (may be NULL) the output before normalising. */
int mm_fno_predict(mm_fno* f, const float* x, int batch, float* m_out, float* raw_out);

/* Synchronise and report whether a tensor-core product gave up waiting (MM_ETIMEOUT). */
int mm_fno_status(mm_fno* f);
const char* mm_fno_last_error(const mm_fno* f);
void mm_fno_destroy(mm_fno* f);

/*
 * The tensor-core product alone:  C[b] = alpha * A[b] B[b]^T  (+ C[b] if beta)
 * for b < batch, A [m][k] and B [n][k] bf16 row-major (k contiguous), C [m][n]
 * fp32 row-major; leading dimensions and batch strides in elements
 * (lda, ldb and the A/B batch strides multiples of 8, base addresses 16-byte
 * aligned).  Asynchronous on cuda_stream; MM_EINVAL for bad strides or
 * alignment.  mm_gemm_status synchronises the stream and returns MM_ETIMEOUT
 * (then clears it) if a product gave up waiting for its operands since the
 * last call.
 */
int mm_gemm_bf16(const void* a, long long lda, long long a_batch, const void* b, long long ldb, long long b_batch,
                 float* c, long long ldc, long long c_batch, int m, int n, int k, int batch, float alpha, int beta,
                 void* cuda_stream);
int mm_gemm_status(void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif
