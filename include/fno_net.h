/*
 * fno_net.h -- C ABI of the fused tensor-core (tcgen05) kernels of the warm-start
 * network: the Fourier neural operator of fno.h (lift, four spectral layers with a
 * pointwise channel mix, GELU, projection; MSE loss), trained and evaluated with BF16
 * activations in device memory and FP32 accumulation in tensor memory.
 *
 * The paper has no counterpart: the network only proposes the initial field of the
 * lattice Boltzmann iteration (lbm.h), which always runs to convergence from it.
 *
 * Network (channels-last, pixel p = (b, r, z), row R = (b, r); C = width, M = modes):
 *   h0 = x P + p                                     lift (in_ch -> C)
 *   pre_l = h_l W_l + b_l + izDFT(V_l),  V_l = irDFT(mix(rDFT(zDFT(h_l)), R_l))
 *   h_{l+1} = GELU(pre_l) (l < L - 1),  h_L = pre_{L-1}
 *   q = GELU(h_L Q1 + q1),  y = q Q2 + q2,  loss = mean (y - t)^2
 * The z transform keeps kz in [0, M) (2M real coefficients: M cosines then M sines, the
 * "kz2" index), the r transform kr in [0, M) U [nr - M, nr) (2M complex modes).
 *
 * Layouts (device memory, row-major, innermost last):
 *   activations h, pre, dpre, dh             BF16 [batch][nr][nz][C]
 *   z-spectra Z, V, dV, dZ                   BF16 [batch][M][2][nr][C]   (kz, re/im, r, c)
 *   k-spectra W, Y, dY, dW                   FP32 [M][2M][2][batch][C]   (kz, kr, re/im, b, c)
 *   spectral weights R                       FP32 [2M][M][C][C][2]       (kr, kz, c_in, c_out, re/im)
 *   operand images (fno_net_pack)            BF16, the tensor-core tile layout of tc.cuh
 * Supported sizes (fno_net_supported): C in {32, 64}; nz a multiple of 128, <= 512;
 * nr a multiple of 128 / C, 2M <= nr, 2 M a multiple of 16, 4 M <= 128; hidden = 128;
 * in_ch <= 16; out_ch <= 16.
 *
 * Every call is asynchronous on `stream` and returns 0, FNO_NET_ERR_INVALID (bad
 * argument) or FNO_NET_ERR_CUDA (launch failure); fno_net_last_error() gives the message.
 * No call allocates device memory.  Gradients are added to the caller's FP32 buffers:
 * each CTA sums its share in tensor or shared memory and adds the sum with FP32 atomics
 * (the order of those additions, and so the last bits of a gradient, may vary from run
 * to run).
 */
#ifndef FNO_NET_H
#define FNO_NET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FNO_NET_OK 0
#define FNO_NET_ERR_INVALID 1
#define FNO_NET_ERR_CUDA 2

typedef struct fno_net_dims {
    int32_t batch, nr, nz, width, modes, hidden, in_ch, out_ch;
} fno_net_dims;

/* 1 if the fused kernels cover these sizes, else 0. */
int fno_net_supported(const fno_net_dims *d);

/* Operand image (BF16, tc.cuh layout) of an FP32 matrix: element (outer o, inner i) =
 * src[o * so + i * si] for o < O, i < I, zero for o < Opad, i < Ipad outside it.
 * Opad and Ipad multiples of 8. */
int fno_net_pack(const float *src, int64_t so, int64_t si, int O, int I, void *dst, int Opad, int Ipad,
                 void *stream);

/* Up to FNO_NET_PACK_MAX fno_net_pack jobs in one launch; `jobs` is host memory (copied
 * into the launch), the pointers in it device memory. */
#define FNO_NET_PACK_MAX 16
typedef struct fno_net_pack_job {
    const float *src;
    int64_t so, si;
    int32_t O, I, Opad, Ipad;
    void *dst;
} fno_net_pack_job;
int fno_net_pack_many(const fno_net_pack_job *jobs, int n, void *stream);

/* Forward pixel kernels, one CTA per group of 128 / C rows, nz / 128 tiles of 128 z each.
 * mode 0 (lift):  out = x P + p (x FP32 [batch][nr][nz][in_ch]; w_img = image of P^T,
 *                 outer C, inner 16); Z = zDFT(out).
 * mode 1 (layer): out = pre = h W + b + izDFT(V) (w_img: image of W^T, outer C, inner C);
 *                 hout = GELU(pre); Z = zDFT(hout).
 * mode 2 (last):  out = h W + b + izDFT(V); no GELU, no Z.
 * gzt_img: image of Gz^T (outer nz, inner 2M), the inverse z transform with its one-sided
 * weights and 1 / (nr nz); fz_img: image of Fz (outer nz, inner 2M), the forward one. */
int fno_net_fwd(int mode, const fno_net_dims *d, const float *x, const void *h, const void *w_img,
                const float *bias, const void *gzt_img, const void *fz_img, const void *V, void *out, void *hout,
                void *Z, void *stream);

/* Projection, one CTA per SM over tiles of 128 pixels: q = GELU(hL Q1 + q1), y = q Q2 + q2.
 * With t != NULL also the loss and the projection's backward: *loss (device double) +=
 * sum (y - t)^2 / (P out_ch); dhL = dL/dhL (BF16); dL/dQ1 ([C][hidden]), dL/dq1, dL/dQ2
 * ([hidden][out_ch]) and dL/dq2 added to dQ1, dq1, dQ2, dq2.  Images: q1w (Q1^T: outer
 * hidden, inner C), q1n (Q1: outer C, inner hidden), q2w (Q2^T: outer 16, inner hidden),
 * q2n (Q2: outer hidden, inner 16). */
int fno_net_proj(const fno_net_dims *d, const void *hL, const void *q1w, const void *q1n, const float *q1,
                 const void *q2w, const void *q2n, const float *q2, const float *t, float *y, void *dhL,
                 double *loss, float *dQ1, float *dq1, float *dQ2, float *dq2, void *stream);

/* Backward pixel kernels (one CTA per SM over row groups).
 * mode 0 (last layer):  dpre = dpre_in (= dL/dh_L); dV = izDFT^T(dpre) (BF16 z-spectrum);
 *                       dL/dW = h^T dpre ([C][C]) and dL/db added to dW, db.
 * mode 1 (layer l > 0): dh = dpre_in W^T + zDFT^T(dZ) (dpre_in = dL/dpre_l, dZ the
 *                       z-spectrum gradient of layer l, wn_img = image of W_l: outer C
 *                       (c_in), inner C (c_out)); dpre_out = dh * GELU'(pre) (pre = pre_{l-1}),
 *                       then as mode 0 with h = h_{l-1} for layer l - 1.
 * mode 2 (layer 0):     dh0 = dpre_in W_0^T + zDFT^T(dZ); dL/dP = x^T dh0 ([in_ch][C], x
 *                       FP32) and dL/dp added to dW, db. */
int fno_net_bwd(int mode, const fno_net_dims *d, const void *dpre_in, const void *dZ, const void *wn_img,
                const void *fz_img, const void *pre, const void *h, const float *x, const void *gzt_img,
                void *dpre_out, void *dV, float *dW, float *db, void *stream);

/* r transforms of one z-spectrum per (batch, kz):
 * fno_net_r2k: out (k-spectrum, FP32) = F2 in (in: BF16 z-spectrum), F2 = [[Cr, Sr], [-Sr, Cr]]
 *   (the forward transform of Z, and the adjoint of the inverse transform for dV);
 * fno_net_k2r: out (BF16 z-spectrum) = F2i in (in: FP32 k-spectrum), F2i = [[Ci, -Si], [Si, Ci]]
 *   (the inverse transform of Y, and the adjoint of the forward one for dW).
 * f2_img: image of F2 (outer 128 rows, rows >= 4M zero; inner 2 nr); f2i_img: image of F2i
 * (outer 2 nr, inner 4M). */
int fno_net_r2k(const fno_net_dims *d, const void *in, const void *f2_img, float *out, void *stream);
int fno_net_k2r(const fno_net_dims *d, const float *in, const void *f2i_img, void *out, void *stream);

/* Per-mode complex channel mixing Y = W R (each (kr, kz): [batch][C] x [C][C]) and its
 * backward: dW = dY R^H (overwritten), dR (+)= W^H dY summed over the batch
 * (accumulate = 1 adds). */
int fno_net_mix_fwd(const fno_net_dims *d, const float *W, const float *R, float *Y, void *stream);
int fno_net_mix_bwd(const fno_net_dims *d, const float *W, const float *R, const float *dY, float *dW, float *dR,
                    int accumulate, void *stream);

/* Status of the bounded tensor-core waits, synchronous: 0 none ran out since the last
 * clear, 1 one ran out (that launch's output is invalid; each CTA waited for its issued
 * MMAs before freeing tensor memory), 2 a recovery wait ran out as well; -1 CUDA error.
 * clear = 1 resets the flag. */
int fno_net_status(int clear);

const char *fno_net_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FNO_NET_H */
