// fno.cu - the learned relaxation warm start: a Fourier neural operator on
// 128 x 128 films, trained and evaluated with BF16 operands and FP32
// accumulation on the tensor cores (tc_gemm.cu).
//
// The paper relaxes a start state with the solver (Sec. 4, Sec. 6 relax());
// the warm start predicts a relaxed state from the film's material and field,
// and the solver finishes the relaxation from there.  The operator (Li et al.,
// ICLR 2021): lift 16 -> 32 channels; four layers z = S(v) + Wp v + b with
// v' = gelu(z) (no gelu after the last); projection 32 -> 128 (gelu) -> 3.
// S(v) keeps 16 modes per axis and sign (512 modes) of the 2-D transform and
// mixes the 32 channels of each kept mode with a complex 32 x 32 matrix.
//
// Every product runs on the tensor cores:
//   * the truncated 2-D transforms are dense products with a DFT basis
//     (forward: [B*32, 16384] x [1024, 16384]^T; inverse: [B*32, 1024] x
//     [16384, 1024]^T), the basis split into two bf16 terms hi + lo so that
//     the transform itself is accurate to ~2^-16;
//   * the mode mixing is a batch of 512 products [B, 64] x [64, 64]^T (the
//     complex 32 x 32 matrix as the real matrix [[Re, -Im], [Im, Re]]);
//   * the point-wise channel maps are [B*16384, Cin] x [Cout, Cin]^T;
//   * weight gradients are products over the batch's cells.
// Activations are stored in bf16 in two layouts (channels-first for the
// transforms, channels-last for the point-wise maps); pre-activations in fp32.
#include "mm.h"
#include "mm_fno.h"
#include "mm_internal.cuh"

#include <cuda_bf16.h>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

namespace {

constexpr int N = 128, NP = N * N, W = 32, NM = 512, MR = 2 * NM, CIN = 16, CH = 128, CO = 3, COP = 16;
typedef __nv_bfloat16 bf16;

// ---- flat parameter layout (fp32 master copy, gradients, Adam moments) -----
constexpr long long P_LIFT_W = 0;                          // [32][16]
constexpr long long P_LIFT_B = P_LIFT_W + W * CIN;         // [32]
constexpr long long P_SPEC = P_LIFT_B + W;                 // [4][2 (re, im)][512][32 out][32 in]
constexpr long long SPEC_L = 2LL * NM * W * W;
constexpr long long P_PW_W = P_SPEC + 4 * SPEC_L;          // [4][32][32]
constexpr long long P_PW_B = P_PW_W + 4 * W * W;           // [4][32]
constexpr long long P_P1_W = P_PW_B + 4 * W;               // [128][32]
constexpr long long P_P1_B = P_P1_W + CH * W;              // [128]
constexpr long long P_P2_W = P_P1_B + CH;                  // [3][128]
constexpr long long P_P2_B = P_P2_W + CO * CH;             // [3]
constexpr long long P_TOTAL = P_P2_B + CO;

size_t a256(size_t v) { return (v + 255) & ~size_t(255); }

// kept mode m = ix*32 + jy -> (ky, kx)
__host__ __device__ inline void mode_k(int m, int& ky, int& kx) {
    kx = m >> 5;
    const int jy = m & 31;
    ky = jy < 16 ? jy : N - 32 + jy;
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// ---- DFT bases (once per workspace) ---------------------------------------
// fb[2m + r][p] = (cos t, -sin t)[r], ib[p][2m + r] = (w(kx)/N^2) (cos t, -sin t)[r],
// t = 2 pi (ky y + kx x)/N, each split as hi + lo bf16
__global__ void k_bases(bf16* fb_hi, bf16* fb_lo, bf16* ib_hi, bf16* ib_lo) {
    const long long total = (long long)MR * NP;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i / NP), p = (int)(i % NP);
        const int m = j >> 1, r = j & 1;
        int ky, kx;
        mode_k(m, ky, kx);
        const int y = p / N, x = p % N;
        const int ph = (ky * y + kx * x) & (N - 1);              // exact phase in units of 2 pi / N
        double s, c;
        sincospi(2.0 * ph / N, &s, &c);
        const double v = r == 0 ? c : -s;
        const bf16 h = __double2bfloat16(v);
        const bf16 l = __double2bfloat16(v - (double)__bfloat162float(h));
        fb_hi[(long long)j * NP + p] = h;
        fb_lo[(long long)j * NP + p] = l;
        const double vi = v * (kx == 0 ? 1.0 : 2.0) / (double)NP;       // exact power-of-two scaling
        const bf16 hi2 = __double2bfloat16(vi);
        const bf16 lo2 = __double2bfloat16(vi - (double)__bfloat162float(hi2));
        ib_hi[(long long)p * MR + j] = hi2;
        ib_lo[(long long)p * MR + j] = lo2;
    }
}

// ---- weights: fp32 master -> bf16 operand copies ----------------------------
struct WPtr {
    bf16 *lift_w, *rf, *rt, *pw, *pwt, *p1, *p1t, *p2, *p2t;
};
__global__ void k_weights_bf16(const float* __restrict__ P, WPtr w) {
    const long long nspec = 4LL * NM * 64 * 64;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nspec;
         i += (long long)gridDim.x * blockDim.x) {
        // rf[l][m][a][b] (a = out index of the real form, b = in index): [[Rr, -Ri], [Ri, Rr]]
        const int b = (int)(i & 63), a = (int)((i >> 6) & 63);
        const long long lm = i >> 12;
        const int l = (int)(lm / NM), m = (int)(lm % NM);
        const int o = a & 31, ii = b & 31;
        const float* re = P + P_SPEC + l * SPEC_L + ((long long)m * W + o) * W + ii;
        const float rr = re[0], ri = re[(long long)NM * W * W];
        float v;
        if (a < 32) v = b < 32 ? rr : -ri;
        else v = b < 32 ? ri : rr;
        w.rf[i] = __float2bfloat16(v);
        // transpose of the real form: rt[l][m][b][a]
        w.rt[(lm << 12) + ((long long)b << 6) + a] = __float2bfloat16(v);
    }
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < W * CIN) w.lift_w[t] = __float2bfloat16(P[P_LIFT_W + t]);
    if (t < 4 * W * W) {
        const int l = t / (W * W), o = (t / W) % W, ii = t % W;
        const float v = P[P_PW_W + t];
        w.pw[t] = __float2bfloat16(v);
        w.pwt[l * W * W + ii * W + o] = __float2bfloat16(v);
    }
    if (t < CH * W) {
        const int j = t / W, ii = t % W;
        const float v = P[P_P1_W + t];
        w.p1[t] = __float2bfloat16(v);
        w.p1t[ii * CH + j] = __float2bfloat16(v);
    }
    if (t < CH * COP) {
        // p2 [3][128] and its transpose padded to [128][16]
        const int j = t / COP, c = t % COP;
        const float v = c < CO ? P[P_P2_W + c * CH + j] : 0.0f;
        w.p2t[j * COP + c] = __float2bfloat16(v);
        if (c < CO) w.p2[c * CH + j] = __float2bfloat16(v);
    }
}

// ---- input features: fp32 [B][16][NP] -> bf16 channels-first and -last ----
__global__ void k_input(const float* __restrict__ x, bf16* xcf, bf16* xcl, int B) {
    const long long total = (long long)B * NP;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / NP, p = i % NP;
#pragma unroll
        for (int c = 0; c < CIN; ++c) {
            const bf16 v = __float2bfloat16(x[(b * CIN + c) * NP + p]);
            xcf[(b * CIN + c) * NP + p] = v;
            xcl[i * CIN + c] = v;
        }
    }
}

// ---- channels-last fp32 C + bias -> (optional gelu) -> bf16 in both layouts
// One block: 32 cells x 32 channels through a shared-memory tile.  cl: [B*NP][C],
// cf: [B][C][NP].  pre (optional) keeps the fp32 pre-activation (cl layout).
__global__ void k_cl_epilogue(const float* in, const float* __restrict__ bias, int C, int act,
                              float* pre, bf16* out_cl, bf16* out_cf, int B) {
    __shared__ float tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;          // 32 x 8
    const long long ntile = (long long)B * (NP / 32) * (C / 32);
    for (long long t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int cb = (int)(t % (C / 32));
        const long long pt = t / (C / 32);
        const long long b = pt / (NP / 32);
        const int p0 = (int)(pt % (NP / 32)) * 32;
        const int c = cb * 32 + tx;
        for (int r = ty; r < 32; r += 8) {
            const long long row = b * NP + p0 + r;
            float v = in[row * C + c] + bias[c];
            if (pre) pre[row * C + c] = v;
            if (act) v = gelu_f(v);
            const bf16 h = __float2bfloat16(v);
            out_cl[row * C + c] = h;
            tile[r][tx] = __bfloat162float(h);
        }
        __syncthreads();
        for (int r = ty; r < 32; r += 8) {
            const int cc = cb * 32 + r;
            out_cf[(b * C + cc) * NP + p0 + tx] = __float2bfloat16(tile[tx][r]);
        }
        __syncthreads();
    }
}

// layer epilogue: z = U (cf) + Wv (cl) + bias; v' = gelu(z) (act) or z
__global__ void k_layer_epilogue(const float* __restrict__ U, const float* __restrict__ Wv,
                                 const float* __restrict__ bias, int act, float* zout, bf16* vcf, bf16* vcl, int B) {
    __shared__ float tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const long long ntile = (long long)B * (NP / 32);
    for (long long t = blockIdx.x; t < ntile; t += gridDim.x) {
        const long long b = t / (NP / 32);
        const int p0 = (int)(t % (NP / 32)) * 32;
        for (int r = ty; r < 32; r += 8) tile[r][tx] = Wv[(b * NP + p0 + r) * W + tx];      // [cell][channel]
        __syncthreads();
        for (int r = ty; r < 32; r += 8) {                 // r = channel, tx = cell
            const long long i = (b * W + r) * NP + p0 + tx;
            const float z = U[i] + tile[tx][r] + bias[r];
            zout[i] = z;
            const bf16 h = __float2bfloat16(act ? gelu_f(z) : z);
            vcf[i] = h;
            tile[tx][r] = __bfloat162float(h);
        }
        __syncthreads();
        for (int r = ty; r < 32; r += 8) vcl[(b * NP + p0 + r) * W + tx] = __float2bfloat16(tile[r][tx]);
        __syncthreads();
    }
}

// forward: Xhat [b][i][2m+r] fp32 -> Xm [m][b][r*32+i] and XmT [m][r*32+i][b] (bf16)
__global__ void k_perm_fwd(const float* __restrict__ X, bf16* Xm, bf16* XmT, int B) {
    const long long total = (long long)B * W * MR;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t % MR);
        const long long bi = t / MR;
        const int i = (int)(bi % W), b = (int)(bi / W);
        const int m = j >> 1, r = j & 1;
        const bf16 v = __float2bfloat16(X[t]);
        Xm[((long long)m * B + b) * 64 + r * 32 + i] = v;
        XmT[((long long)m * 64 + r * 32 + i) * B + b] = v;
    }
}
// forward: Ym [m][b][r*32+o] fp32 -> Yhat [b][o][2m+r] bf16
__global__ void k_perm_mid(const float* __restrict__ Y, bf16* Yhat, int B) {
    const long long total = (long long)B * W * MR;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t % MR);
        const long long bo = t / MR;
        const int o = (int)(bo % W), b = (int)(bo / W);
        const int m = j >> 1, r = j & 1;
        Yhat[t] = __float2bfloat16(Y[((long long)m * B + b) * 64 + r * 32 + o]);
    }
}
// backward: G [b][o][2m+r] fp32 (rfft of dz) -> dYm [m][b][r*32+o], dYmT [m][r*32+o][b],
// scaled by w(kx)/N^2
__global__ void k_perm_bwd1(const float* __restrict__ G, bf16* dYm, bf16* dYmT, int B) {
    const long long total = (long long)B * W * MR;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t % MR);
        const long long bo = t / MR;
        const int o = (int)(bo % W), b = (int)(bo / W);
        const int m = j >> 1, r = j & 1;
        const float s = ((m >> 5) == 0 ? 1.0f : 2.0f) / (float)NP;
        const bf16 v = __float2bfloat16(G[t] * s);
        dYm[((long long)m * B + b) * 64 + r * 32 + o] = v;
        dYmT[((long long)m * 64 + r * 32 + o) * B + b] = v;
    }
}
// backward: dXm [m][b][r*32+i] fp32 -> dVhat [b][i][2m+r] bf16, scaled by N^2/w(kx)
__global__ void k_perm_bwd2(const float* __restrict__ dX, bf16* dV, int B) {
    const long long total = (long long)B * W * MR;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t % MR);
        const long long bi = t / MR;
        const int i = (int)(bi % W), b = (int)(bi / W);
        const int m = j >> 1, r = j & 1;
        const float s = (float)NP / ((m >> 5) == 0 ? 1.0f : 2.0f);
        dV[t] = __float2bfloat16(dX[((long long)m * B + b) * 64 + r * 32 + i] * s);
    }
}

// projection output: out = C (cl, ldc 4) + q2.  Training: loss sum, dout = 2 (out - tgt)/nel
// in bf16 (cl [B*NP][16], cf [B][16][NP], padding channels zero).  Prediction: m = out/|out|.
__global__ void k_out(const float* __restrict__ C, const float* __restrict__ q2, const float* __restrict__ tgt,
                      float inv_nel, double* loss, bf16* dcl, bf16* dcf, float* m_out, float* raw_out, int B) {
    const long long total = (long long)B * NP;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / NP, p = i % NP;
        float o[CO];
#pragma unroll
        for (int c = 0; c < CO; ++c) o[c] = C[i * 4 + c] + q2[c];
        if (raw_out) {
#pragma unroll
            for (int c = 0; c < CO; ++c) raw_out[(b * CO + c) * NP + p] = o[c];
        }
        if (m_out) {
            const float nrm = sqrtf(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]);
            const float inv = nrm > 0.f ? 1.0f / nrm : 0.f;
#pragma unroll
            for (int c = 0; c < CO; ++c) m_out[(b * CO + c) * NP + p] = nrm > 0.f ? o[c] * inv : (c == 0 ? 1.f : 0.f);
        }
        if (tgt) {
#pragma unroll
            for (int c = 0; c < COP; ++c) {
                float d = 0.f;
                if (c < CO) {
                    const float e = o[c] - tgt[(b * CO + c) * NP + p];
                    acc += (double)e * (double)e;
                    d = 2.0f * e * inv_nel;
                }
                const bf16 h = __float2bfloat16(d);
                dcl[i * COP + c] = h;
                dcf[(b * COP + c) * NP + p] = h;
            }
        }
    }
    if (tgt) {
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
    }
}

// dz = (dv_cf + dv_cl) * (act ? gelu'(z) : 1) -> bf16 cf and cl; bias gradient sum
// (C = 32 or 128 channels; dv_cf may be null; z_cf (act) is channels-first,
// z_cl (act, projection) channels-last - exactly one of them is used)
__global__ void k_dz(const float* __restrict__ dv_cf, const float* __restrict__ dv_cl, const float* __restrict__ z_cf,
                     const float* __restrict__ z_cl, int C, int act, bf16* dz_cf, bf16* dz_cl, float* dbias, int B) {
    __shared__ float tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ncb = C / 32;
    const long long ntile = (long long)B * (NP / 32) * ncb;
    float part = 0.f;          // bias partial of channel cb*32 + tx (per thread, in the cl pass)
    int cb_last = -1;
    for (long long t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int cb = (int)(t % ncb);
        const long long pt = t / ncb;
        const long long b = pt / (NP / 32);
        const int p0 = (int)(pt % (NP / 32)) * 32;
        if (cb != cb_last) {
            if (cb_last >= 0) atomicAdd(&dbias[cb_last * 32 + tx], part);
            part = 0.f;
            cb_last = cb;
        }
        // channels-last pass: tx = channel, rows = cells
        for (int r = ty; r < 32; r += 8) {
            const long long row = b * NP + p0 + r;
            const int c = cb * 32 + tx;
            float d = dv_cl[row * C + c];
            if (dv_cf) d += dv_cf[(b * C + c) * NP + p0 + r];
            if (act) d *= gelu_grad_f(z_cf ? z_cf[(b * C + c) * NP + p0 + r] : z_cl[row * C + c]);
            const bf16 h = __float2bfloat16(d);
            dz_cl[row * C + c] = h;
            const float hv = __bfloat162float(h);
            part += hv;
            tile[r][tx] = hv;
        }
        __syncthreads();
        for (int r = ty; r < 32; r += 8) dz_cf[(b * C + cb * 32 + r) * NP + p0 + tx] = __float2bfloat16(tile[tx][r]);
        __syncthreads();
    }
    if (cb_last >= 0) atomicAdd(&dbias[cb_last * 32 + tx], part);
}

// bias gradient of the projection output (channels 0..2 of dcl [B*NP][16])
__global__ void k_bias_out(const bf16* __restrict__ dcl, float* dq2, int B) {
    float s[CO] = {0.f, 0.f, 0.f};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)B * NP;
         i += (long long)gridDim.x * blockDim.x)
        for (int c = 0; c < CO; ++c) s[c] += __bfloat162float(dcl[i * COP + c]);
    for (int c = 0; c < CO; ++c) {
        float v = s[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&dq2[c], v);
    }
}

// dR' [m][64 out][64 in] -> gradient of the complex weights (re, im planes)
__global__ void k_dR(const float* __restrict__ dR, float* g_spec) {
    const long long total = (long long)NM * W * W;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % W), o = (int)((t / W) % W);
        const long long m = t / (W * W);
        const float* d = dR + m * 4096;
        g_spec[t] = d[o * 64 + i] + d[(32 + o) * 64 + 32 + i];
        g_spec[(long long)NM * W * W + t] = d[(32 + o) * 64 + i] - d[o * 64 + 32 + i];
    }
}

// sum over the batch of per-sample products (row stride ldp, batch stride bstride)
// -> grad [rows][cols]
__global__ void k_sum_batch(const float* __restrict__ part, int B, int rows, int cols, int ldp, long long bstride,
                            float* g) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * cols) return;
    const int r = t / cols, c = t % cols;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += part[b * bstride + (long long)r * ldp + c];
    g[t] = s;
}

__global__ void k_adam(float* P, const float* __restrict__ G, float* M1, float* M2, long long n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float g = G[i];
        const float m = b1 * M1[i] + (1.f - b1) * g;
        const float v = b2 * M2[i] + (1.f - b2) * g * g;
        M1[i] = m;
        M2[i] = v;
        P[i] -= lr * (m * c1) / (sqrtf(v * c2) + eps);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
struct mm_fno {
    int max_batch = 0;
    cudaStream_t stream = nullptr;
    char* ws = nullptr;
    size_t total = 0;
    std::string err;
    long long step = 0;
    bool ready = false;
    // buffers
    float *P = nullptr, *G = nullptr, *M1 = nullptr, *M2 = nullptr;
    bf16 *fb_hi, *fb_lo, *ib_hi, *ib_lo;
    WPtr w;
    bf16 *xcf, *xcl;
    bf16 *vcf[5], *vcl[5];
    float* z[4];
    bf16 *Xm[4], *XmT[4];
    float *Xhat, *Ym, *U, *Wv;
    bf16* Yhat;
    float* hp;
    bf16 *hcl, *hcf;
    float* outc;
    bf16 *dcl, *dcf;
    float *dh, *dvcl, *dvcf;
    bf16 *dzcl, *dzcf;                 // sized for 128 channels (reused for 32)
    bf16 *dYm, *dYmT, *dV;
    float *dR, *dXm;
    float* part;                       // per-sample weight-gradient products
    double* loss;
    unsigned* errw;
};

namespace {

int fail(mm_fno* f, int code, const char* msg) {
    if (f) f->err = msg;
    return code;
}
#define FCK(call)                                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            if (f) f->err = std::string(#call) + ": " + cudaGetErrorString(e_);        \
            return MM_ECUDA;                                                           \
        }                                                                              \
    } while (0)

int grid_for(long long n, int per = 256) {
    long long g = (n + per - 1) / per;
    return (int)(g < 4 * 152 ? (g < 1 ? 1 : g) : 4 * 152);
}

void layout(mm_fno* f, char* base) {
    const long long B = f->max_batch;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base ? base + off : nullptr;
        off += a256(bytes);
        return p;
    };
    f->P = (float*)take(P_TOTAL * 4);
    f->G = (float*)take(P_TOTAL * 4);
    f->M1 = (float*)take(P_TOTAL * 4);
    f->M2 = (float*)take(P_TOTAL * 4);
    f->fb_hi = (bf16*)take((size_t)MR * NP * 2);
    f->fb_lo = (bf16*)take((size_t)MR * NP * 2);
    f->ib_hi = (bf16*)take((size_t)MR * NP * 2);
    f->ib_lo = (bf16*)take((size_t)MR * NP * 2);
    f->w.lift_w = (bf16*)take(W * CIN * 2);
    f->w.rf = (bf16*)take(4LL * NM * 4096 * 2);
    f->w.rt = (bf16*)take(4LL * NM * 4096 * 2);
    f->w.pw = (bf16*)take(4 * W * W * 2);
    f->w.pwt = (bf16*)take(4 * W * W * 2);
    f->w.p1 = (bf16*)take(CH * W * 2);
    f->w.p1t = (bf16*)take(CH * W * 2);
    f->w.p2 = (bf16*)take(CO * CH * 2);
    f->w.p2t = (bf16*)take(CH * COP * 2);
    f->xcf = (bf16*)take(B * CIN * NP * 2);
    f->xcl = (bf16*)take(B * CIN * NP * 2);
    for (int l = 0; l < 5; ++l) {
        f->vcf[l] = (bf16*)take(B * W * NP * 2);
        f->vcl[l] = (bf16*)take(B * W * NP * 2);
    }
    for (int l = 0; l < 4; ++l) {
        f->z[l] = (float*)take(B * W * NP * 4);
        f->Xm[l] = (bf16*)take(B * W * MR * 2);
        f->XmT[l] = (bf16*)take(B * W * MR * 2);
    }
    f->Xhat = (float*)take(B * W * MR * 4);
    f->Ym = (float*)take(B * W * MR * 4);
    f->Yhat = (bf16*)take(B * W * MR * 2);
    f->U = (float*)take(B * W * NP * 4);
    f->Wv = (float*)take(B * W * NP * 4);
    f->hp = (float*)take(B * CH * NP * 4);
    f->hcl = (bf16*)take(B * CH * NP * 2);
    f->hcf = (bf16*)take(B * CH * NP * 2);
    f->outc = (float*)take(B * NP * 4 * 4);
    f->dcl = (bf16*)take(B * NP * COP * 2);
    f->dcf = (bf16*)take(B * NP * COP * 2);
    f->dh = (float*)take(B * CH * NP * 4);
    f->dvcl = (float*)take(B * W * NP * 4);
    f->dvcf = (float*)take(B * W * NP * 4);
    f->dzcl = (bf16*)take(B * CH * NP * 2);
    f->dzcf = (bf16*)take(B * CH * NP * 2);
    f->dYm = (bf16*)take(B * W * MR * 2);
    f->dYmT = (bf16*)take(B * W * MR * 2);
    f->dV = (bf16*)take(B * W * MR * 2);
    f->dR = (float*)take((size_t)NM * 4096 * 4);
    f->dXm = (float*)take(B * W * MR * 4);
    f->part = (float*)take(B * CH * CH * 4);
    f->loss = (double*)take(8);
    f->errw = (unsigned*)take(4);
    f->total = off;
}

// C = alpha A B^T (+C) with the library's tensor-core product
int gemm(mm_fno* f, const bf16* a, long long lda, long long ab, const bf16* b, long long ldb, long long bb, float* c,
         long long ldc, long long cb, int m, int n, int k, int batch, int beta) {
    FCK(mm::gemm_bf16(a, lda, ab, b, ldb, bb, c, ldc, cb, m, n, k, batch, 1.0f, beta, f->errw, f->stream));
    return MM_OK;
}

int forward(mm_fno* f, int B, bool train) {
    int rc;
    cudaStream_t s = f->stream;
    const dim3 tb(32, 8);
    // lift: [B*NP, 16] x [32, 16]^T
    if ((rc = gemm(f, f->xcl, CIN, 0, f->w.lift_w, CIN, 0, f->Wv, W, 0, B * NP, W, CIN, 1, 0))) return rc;
    k_cl_epilogue<<<grid_for((long long)B * NP, 1024), tb, 0, s>>>(f->Wv, f->P + P_LIFT_B, W, 0, nullptr, f->vcl[0],
                                                                   f->vcf[0], B);
    FCK(cudaGetLastError());
    for (int l = 0; l < 4; ++l) {
        // truncated forward transform (basis hi + lo)
        if ((rc = gemm(f, f->vcf[l], NP, 0, f->fb_hi, NP, 0, f->Xhat, MR, 0, B * W, MR, NP, 1, 0))) return rc;
        if ((rc = gemm(f, f->vcf[l], NP, 0, f->fb_lo, NP, 0, f->Xhat, MR, 0, B * W, MR, NP, 1, 1))) return rc;
        k_perm_fwd<<<grid_for((long long)B * W * MR), 256, 0, s>>>(f->Xhat, f->Xm[l], f->XmT[l], B);
        FCK(cudaGetLastError());
        // mode mixing: per mode [B, 64] x [64, 64]^T
        if ((rc = gemm(f, f->Xm[l], 64, (long long)B * 64, f->w.rf + (long long)l * NM * 4096, 64, 4096, f->Ym, 64,
                       (long long)B * 64, B, 64, 64, NM, 0)))
            return rc;
        k_perm_mid<<<grid_for((long long)B * W * MR), 256, 0, s>>>(f->Ym, f->Yhat, B);
        FCK(cudaGetLastError());
        // truncated inverse transform
        if ((rc = gemm(f, f->Yhat, MR, 0, f->ib_hi, MR, 0, f->U, NP, 0, B * W, NP, MR, 1, 0))) return rc;
        if ((rc = gemm(f, f->Yhat, MR, 0, f->ib_lo, MR, 0, f->U, NP, 0, B * W, NP, MR, 1, 1))) return rc;
        // point-wise channel map
        if ((rc = gemm(f, f->vcl[l], W, 0, f->w.pw + l * W * W, W, 0, f->Wv, W, 0, B * NP, W, W, 1, 0))) return rc;
        k_layer_epilogue<<<grid_for((long long)B * NP / 32, 1), tb, 0, s>>>(f->U, f->Wv, f->P + P_PW_B + l * W,
                                                                          l < 3 ? 1 : 0, f->z[l], f->vcf[l + 1],
                                                                          f->vcl[l + 1], B);
        FCK(cudaGetLastError());
    }
    // projection
    if ((rc = gemm(f, f->vcl[4], W, 0, f->w.p1, W, 0, f->hp, CH, 0, B * NP, CH, W, 1, 0))) return rc;
    k_cl_epilogue<<<grid_for((long long)B * NP * 4, 1024), tb, 0, s>>>(f->hp, f->P + P_P1_B, CH, 1, f->hp, f->hcl,
                                                                       f->hcf, B);
    FCK(cudaGetLastError());
    if ((rc = gemm(f, f->hcl, CH, 0, f->w.p2, CH, 0, f->outc, 4, 0, B * NP, CO, CH, 1, 0))) return rc;
    (void)train;
    return MM_OK;
}

int backward(mm_fno* f, int B) {
    int rc;
    cudaStream_t s = f->stream;
    const dim3 tb(32, 8);
    float* G = f->G;
    FCK(cudaMemsetAsync(G, 0, P_TOTAL * 4, s));
    // output layer: dQ2 = sum_b dout_cf[b] [16][NP] x h_cf[b] [128][NP]^T
    if ((rc = gemm(f, f->dcf, NP, (long long)COP * NP, f->hcf, NP, (long long)CH * NP, f->part, CH, (long long)COP * CH,
                   COP, CH, NP, B, 0)))
        return rc;
    k_sum_batch<<<(CO * CH + 255) / 256, 256, 0, s>>>(f->part, B, CO, CH, CH, (long long)COP * CH, G + P_P2_W);
    k_bias_out<<<grid_for((long long)B * NP), 256, 0, s>>>(f->dcl, G + P_P2_B, B);
    // dh = dout_cl [B*NP][16] x p2t [128][16]^T
    if ((rc = gemm(f, f->dcl, COP, 0, f->w.p2t, COP, 0, f->dh, CH, 0, B * NP, CH, COP, 1, 0))) return rc;
    k_dz<<<grid_for((long long)B * NP * 4 / 32, 1), tb, 0, s>>>(nullptr, f->dh, nullptr, f->hp, CH, 1, f->dzcf, f->dzcl,
                                                               G + P_P1_B, B);
    FCK(cudaGetLastError());
    // dQ1 = sum_b dhp_cf[b] [128][NP] x v4_cf[b] [32][NP]^T
    if ((rc = gemm(f, f->dzcf, NP, (long long)CH * NP, f->vcf[4], NP, (long long)W * NP, f->part, W, (long long)CH * W,
                   CH, W, NP, B, 0)))
        return rc;
    k_sum_batch<<<(CH * W + 255) / 256, 256, 0, s>>>(f->part, B, CH, W, W, (long long)CH * W, G + P_P1_W);
    // dv4 = dhp_cl [B*NP][128] x p1t [32][128]^T
    if ((rc = gemm(f, f->dzcl, CH, 0, f->w.p1t, CH, 0, f->dvcl, W, 0, B * NP, W, CH, 1, 0))) return rc;
    bool have_cf = false;
    for (int l = 3; l >= 0; --l) {
        k_dz<<<grid_for((long long)B * NP / 32, 1), tb, 0, s>>>(have_cf ? f->dvcf : nullptr, f->dvcl,
                                                               l < 3 ? f->z[l] : nullptr, nullptr, W, l < 3 ? 1 : 0,
                                                               f->dzcf, f->dzcl, G + P_PW_B + l * W, B);
        FCK(cudaGetLastError());
        // dWp = sum_b dz_cf[b] [32][NP] x v_cf[b] [32][NP]^T
        if ((rc = gemm(f, f->dzcf, NP, (long long)W * NP, f->vcf[l], NP, (long long)W * NP, f->part, W,
                       (long long)W * W, W, W, NP, B, 0)))
            return rc;
        k_sum_batch<<<(W * W + 255) / 256, 256, 0, s>>>(f->part, B, W, W, W, (long long)W * W, G + P_PW_W + l * W * W);
        // point-wise part of dv_l: dz_cl [B*NP][32] x pwt [32][32]^T
        if ((rc = gemm(f, f->dzcl, W, 0, f->w.pwt + l * W * W, W, 0, f->dvcl, W, 0, B * NP, W, W, 1, 0))) return rc;
        // spectral part: G = dz_cf x fb^T (rfft of dz on the kept modes)
        if ((rc = gemm(f, f->dzcf, NP, 0, f->fb_hi, NP, 0, f->Xhat, MR, 0, B * W, MR, NP, 1, 0))) return rc;
        if ((rc = gemm(f, f->dzcf, NP, 0, f->fb_lo, NP, 0, f->Xhat, MR, 0, B * W, MR, NP, 1, 1))) return rc;
        k_perm_bwd1<<<grid_for((long long)B * W * MR), 256, 0, s>>>(f->Xhat, f->dYm, f->dYmT, B);
        FCK(cudaGetLastError());
        // dR' per mode = dYm^T Xm: [64][B] x [64][B]^T
        if ((rc = gemm(f, f->dYmT, B, 64LL * B, f->XmT[l], B, 64LL * B, f->dR, 64, 4096, 64, 64, B, NM, 0))) return rc;
        k_dR<<<grid_for((long long)NM * W * W), 256, 0, s>>>(f->dR, G + P_SPEC + l * SPEC_L);
        FCK(cudaGetLastError());
        // dXm = dYm [B][64] x rt [64 in][64 out]^T per mode
        if ((rc = gemm(f, f->dYm, 64, 64LL * B, f->w.rt + (long long)l * NM * 4096, 64, 4096, f->dXm, 64, 64LL * B, B,
                       64, 64, NM, 0)))
            return rc;
        k_perm_bwd2<<<grid_for((long long)B * W * MR), 256, 0, s>>>(f->dXm, f->dV, B);
        FCK(cudaGetLastError());
        // dv (cf) = dV [B*32][1024] x ib^T
        if ((rc = gemm(f, f->dV, MR, 0, f->ib_hi, MR, 0, f->dvcf, NP, 0, B * W, NP, MR, 1, 0))) return rc;
        if ((rc = gemm(f, f->dV, MR, 0, f->ib_lo, MR, 0, f->dvcf, NP, 0, B * W, NP, MR, 1, 1))) return rc;
        have_cf = true;
    }
    // lift: dv0 (no activation) -> bf16, dWl = sum_b dv0_cf[b] [32][NP] x x_cf[b] [16][NP]^T
    k_dz<<<grid_for((long long)B * NP / 32, 1), tb, 0, s>>>(f->dvcf, f->dvcl, nullptr, nullptr, W, 0, f->dzcf, f->dzcl,
                                                           G + P_LIFT_B, B);
    FCK(cudaGetLastError());
    if ((rc = gemm(f, f->dzcf, NP, (long long)W * NP, f->xcf, NP, (long long)CIN * NP, f->part, CIN,
                   (long long)W * CIN, W, CIN, NP, B, 0)))
        return rc;
    k_sum_batch<<<(W * CIN + 255) / 256, 256, 0, s>>>(f->part, B, W, CIN, CIN, (long long)W * CIN, G + P_LIFT_W);
    FCK(cudaGetLastError());
    return MM_OK;
}

int refresh_weights(mm_fno* f) {
    k_weights_bf16<<<grid_for(4LL * NM * 4096), 256, 0, f->stream>>>(f->P, f->w);
    FCK(cudaGetLastError());
    return MM_OK;
}

int check(mm_fno* f, int batch) {
    if (!f) return MM_EINVAL;
    if (!f->ready) return fail(f, MM_ESTATE, "workspace or weights not set");
    if (batch < 1 || batch > f->max_batch || (batch & 7)) return fail(f, MM_EINVAL, "batch must be a multiple of 8 in [8, max_batch]");
    return MM_OK;
}

}  // namespace

extern "C" {

int mm_fno_create(mm_fno** out, int max_batch, void* cuda_stream) {
    if (!out) return MM_EINVAL;
    *out = nullptr;
    if (max_batch < 8 || max_batch > 1024 || (max_batch & 7)) return MM_EINVAL;
    mm_fno* f = new (std::nothrow) mm_fno();
    if (!f) return MM_ENOMEM;
    f->max_batch = max_batch;
    f->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    layout(f, nullptr);
    *out = f;
    return MM_OK;
}

size_t mm_fno_workspace_bytes(const mm_fno* f) { return f ? f->total : 0; }
size_t mm_fno_param_count(void) { return (size_t)P_TOTAL; }

int mm_fno_set_workspace(mm_fno* f, void* dev_ptr, size_t bytes) {
    if (!f || !dev_ptr) return fail(f, MM_EINVAL, "null workspace");
    if (reinterpret_cast<uintptr_t>(dev_ptr) & 255) return fail(f, MM_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < f->total) return fail(f, MM_ENOMEM, "workspace smaller than mm_fno_workspace_bytes()");
    f->ws = static_cast<char*>(dev_ptr);
    layout(f, f->ws);
    FCK(mm::gemm_configure());
    FCK(cudaMemsetAsync(f->ws, 0, f->total, f->stream));
    k_bases<<<4 * 152, 256, 0, f->stream>>>(f->fb_hi, f->fb_lo, f->ib_hi, f->ib_lo);
    FCK(cudaGetLastError());
    return MM_OK;
}

int mm_fno_set_params(mm_fno* f, const float* params) {
    if (!f || !params) return MM_EINVAL;
    if (!f->ws) return fail(f, MM_ESTATE, "workspace not set");
    FCK(cudaMemcpyAsync(f->P, params, P_TOTAL * 4, cudaMemcpyDeviceToDevice, f->stream));
    FCK(cudaMemsetAsync(f->M1, 0, P_TOTAL * 4, f->stream));
    FCK(cudaMemsetAsync(f->M2, 0, P_TOTAL * 4, f->stream));
    f->step = 0;
    int rc = refresh_weights(f);
    if (rc) return rc;
    f->ready = true;
    return MM_OK;
}

int mm_fno_get_params(mm_fno* f, float* params) {
    if (!f || !params) return MM_EINVAL;
    if (!f->ready) return fail(f, MM_ESTATE, "weights not set");
    FCK(cudaMemcpyAsync(params, f->P, P_TOTAL * 4, cudaMemcpyDeviceToDevice, f->stream));
    return MM_OK;
}

int mm_fno_train_step(mm_fno* f, const float* x, const float* target, int batch, float lr, float beta1, float beta2,
                      float eps, double* loss_host, float* grad_out) {
    int rc = check(f, batch);
    if (rc) return rc;
    if (!x || !target) return fail(f, MM_EINVAL, "null input");
    cudaStream_t s = f->stream;
    k_input<<<grid_for((long long)batch * NP), 256, 0, s>>>(x, f->xcf, f->xcl, batch);
    FCK(cudaGetLastError());
    if ((rc = forward(f, batch, true))) return rc;
    FCK(cudaMemsetAsync(f->loss, 0, 8, s));
    const float inv_nel = 1.0f / (float)((long long)batch * NP * CO);
    k_out<<<grid_for((long long)batch * NP), 256, 0, s>>>(f->outc, f->P + P_P2_B, target, inv_nel, f->loss, f->dcl,
                                                        f->dcf, nullptr, nullptr, batch);
    FCK(cudaGetLastError());
    if ((rc = backward(f, batch))) return rc;
    if (grad_out) FCK(cudaMemcpyAsync(grad_out, f->G, P_TOTAL * 4, cudaMemcpyDeviceToDevice, s));
    if (lr != 0.0f) {
        f->step += 1;
        const float c1 = 1.0f / (1.0f - powf(beta1, (float)f->step));
        const float c2 = 1.0f / (1.0f - powf(beta2, (float)f->step));
        k_adam<<<grid_for(P_TOTAL), 256, 0, s>>>(f->P, f->G, f->M1, f->M2, P_TOTAL, lr, beta1, beta2, eps, c1, c2);
        FCK(cudaGetLastError());
        if ((rc = refresh_weights(f))) return rc;
    }
    if (loss_host) {
        double l = 0.0;
        unsigned e = 0;
        FCK(cudaMemcpyAsync(&l, f->loss, 8, cudaMemcpyDeviceToHost, s));
        FCK(cudaMemcpyAsync(&e, f->errw, 4, cudaMemcpyDeviceToHost, s));
        FCK(cudaStreamSynchronize(s));
        *loss_host = l * inv_nel;
        if (e) return fail(f, MM_ETIMEOUT, "a tensor-core product gave up waiting for its operands");
    }
    return MM_OK;
}

int mm_fno_predict(mm_fno* f, const float* x, int batch, float* m_out, float* raw_out) {
    int rc = check(f, batch);
    if (rc) return rc;
    if (!x) return fail(f, MM_EINVAL, "null input");
    cudaStream_t s = f->stream;
    k_input<<<grid_for((long long)batch * NP), 256, 0, s>>>(x, f->xcf, f->xcl, batch);
    FCK(cudaGetLastError());
    if ((rc = forward(f, batch, false))) return rc;
    k_out<<<grid_for((long long)batch * NP), 256, 0, s>>>(f->outc, f->P + P_P2_B, nullptr, 0.f, nullptr, nullptr,
                                                        nullptr, m_out, raw_out, batch);
    FCK(cudaGetLastError());
    return MM_OK;
}

int mm_fno_status(mm_fno* f) {
    if (!f || !f->ws) return MM_EINVAL;
    unsigned e = 0;
    FCK(cudaMemcpyAsync(&e, f->errw, 4, cudaMemcpyDeviceToHost, f->stream));
    FCK(cudaStreamSynchronize(f->stream));
    return e ? MM_ETIMEOUT : MM_OK;
}

const char* mm_fno_last_error(const mm_fno* f) { return f ? f->err.c_str() : "null context"; }

void mm_fno_destroy(mm_fno* f) { delete f; }

// the tensor-core product alone (its own error word, in the library's static memory)
static __device__ unsigned g_gemm_err;

int mm_gemm_bf16(const void* a, long long lda, long long a_batch, const void* b, long long ldb, long long b_batch,
                 float* c, long long ldc, long long c_batch, int m, int n, int k, int batch, float alpha, int beta,
                 void* cuda_stream) {
    unsigned* err = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&err), g_gemm_err) != cudaSuccess) return MM_ECUDA;
    const cudaError_t e = mm::gemm_bf16(a, lda, a_batch, b, ldb, b_batch, c, ldc, c_batch, m, n, k, batch, alpha,
                                        beta, err, reinterpret_cast<cudaStream_t>(cuda_stream));
    if (e == cudaErrorInvalidValue) return MM_EINVAL;
    return e == cudaSuccess ? MM_OK : MM_ECUDA;
}

int mm_gemm_status(void* cuda_stream) {
    unsigned* err = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&err), g_gemm_err) != cudaSuccess) return MM_ECUDA;
    unsigned e = 0;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    if (cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MM_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MM_ECUDA;
    if (e) {
        const unsigned z = 0;
        cudaMemcpyAsync(err, &z, 4, cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
    }
    return e ? MM_ETIMEOUT : MM_OK;
}

}  // extern "C"
