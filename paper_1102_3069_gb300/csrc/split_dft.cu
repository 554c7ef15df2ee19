// split_dft.cu - the z column pass of 3-D grids as split-BF16 DFT products on
// the tensor cores (a precision variant of the FP32 k_colconv<., 1> pass).
//
// Sec. 3.3 runs the whole convolution in single precision.  This variant
// runs the z transforms of stage (i) and (iii) of Sec. 3.2 as dense DFT
// products with bf16 operands and fp32 accumulation: every operand v is
// split into hi = bf16(v) and lo = bf16(v - hi), and a product is formed
// from three tensor-core products, hi*hi + hi*lo + lo*hi (the lo*lo term,
// ~2^-16 relative, is dropped).  Per line of the y spectrum (component,
// kx, ky; nz valid z, padded length Pz):
//   gather   A[line][2z + r] = (Re, Im)[r] of s2 at z < nz (zeros up to nzp)
//   forward  X = A F^T, F[2k + r'][2z + r] the real form of e^{-2 pi i k z / Pz}
//   product  Y = -K^ X per frequency with the real symmetric kernel (stage ii)
//   inverse  O = Y G^T, G[2z + r][2k + r'] the real form of e^{+2 pi i k z / Pz}
//   scatter  s2 at z < nz = O
#include "mm_internal.cuh"

#include <cuda_bf16.h>

namespace mm {
namespace {

typedef __nv_bfloat16 bf16;

size_t a256(size_t v) { return (v + 255) & ~size_t(255); }

__device__ __forceinline__ void split_store(bf16* hi, bf16* lo, long long i, float v) {
    const bf16 h = __float2bfloat16(v);
    hi[i] = h;
    lo[i] = __float2bfloat16(v - __bfloat162float(h));
}

__global__ void k_zs_tables(int pz, int nz, int kp, bf16* f_hi, bf16* f_lo, bf16* g_hi, bf16* g_lo) {
    const int n2 = 2 * pz;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n2 * kp; t += gridDim.x * blockDim.x) {
        const int row = t / kp, col = t % kp;          // F: row = 2k + r', col = 2z + r
        {
            const int k = row >> 1, rr = row & 1, z = col >> 1, r = col & 1;
            double v = 0.0;
            if (z < nz) {
                double s, c;
                sincospi(2.0 * (double)((long long)k * z % pz) / pz, &s, &c);
                // (a + ib)(c - is): re = a c + b s, im = b c - a s
                v = rr == 0 ? (r == 0 ? c : s) : (r == 0 ? -s : c);
            }
            const bf16 h = __double2bfloat16(v);
            f_hi[t] = h;
            f_lo[t] = __double2bfloat16(v - (double)__bfloat162float(h));
        }
        {
            // G: row = 2z + r (kp rows), col = 2k + r' (n2 columns); same t range
            const int grow = t / n2, gcol = t % n2;
            const int z = grow >> 1, r = grow & 1, k = gcol >> 1, rr = gcol & 1;
            double v = 0.0;
            if (z < nz) {
                double s, c;
                sincospi(2.0 * (double)((long long)k * z % pz) / pz, &s, &c);
                // (a + ib)(c + is): re = a c - b s, im = a s + b c
                v = r == 0 ? (rr == 0 ? c : -s) : (rr == 0 ? s : c);
            }
            const bf16 h = __double2bfloat16(v);
            g_hi[t] = h;
            g_lo[t] = __double2bfloat16(v - (double)__bfloat162float(h));
        }
    }
}

__global__ void k_zs_gather(HotParams p, LaunchArgs a) {
    if (a.mode != LM_EVAL && p.st->done) return;
    const long long lines = 3LL * p.hx * p.py;
    const int kp = p.zs_kp, nzp = p.nzp;
    bf16* hi = static_cast<bf16*>(p.zs_a_hi);
    bf16* lo = static_cast<bf16*>(p.zs_a_lo);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < lines * nzp;
         t += (long long)gridDim.x * blockDim.x) {
        const long long l = t / nzp;
        const int z = (int)(t % nzp);
        float2 v = make_float2(0.f, 0.f);
        if (z < p.nz) v = p.s2[l * nzp + z];
        split_store(hi, lo, l * kp + 2 * z, v.x);
        split_store(hi, lo, l * kp + 2 * z + 1, v.y);
    }
}

// Y = K^ X for the three components of column (kx, ky) at frequency k
__global__ void k_zs_product(HotParams p, LaunchArgs a) {
    if (a.mode != LM_EVAL && p.st->done) return;
    const int HX = p.hx, PY = p.py, PZ = p.pz, n2 = 2 * PZ;
    const long long cols = (long long)HX * PY;
    const long long cs = (long long)HX * p.hyk * p.hzk;
    bf16* yhi = static_cast<bf16*>(p.zs_y_hi);
    bf16* ylo = static_cast<bf16*>(p.zs_y_lo);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < cols * PZ;
         t += (long long)gridDim.x * blockDim.x) {
        const long long col = t / PZ;
        const int k = (int)(t % PZ);
        const int kx = (int)(col / PY), ky = (int)(col % PY);
        const bool hi = k > (PZ >> 1);
        const int kq = hi ? PZ - k : k;
        const bool yh = ky > (PY >> 1);
        const int kyq = yh ? PY - ky : ky;
        const long long b = ((long long)kx * p.hyk + kyq) * p.hzk + kq;
        const float kxx = p.kt[b], kyy = p.kt[cs + b], kzz = p.kt[2 * cs + b];
        float kxy = p.kt[3 * cs + b], kxz = p.kt[4 * cs + b], kyz = p.kt[5 * cs + b];
        if (yh) { kxy = -kxy; kyz = -kyz; }
        if (hi) { kxz = -kxz; kyz = -kyz; }
        long long row[3];
        float2 X[3];
        for (int c = 0; c < 3; ++c) {
            row[c] = ((long long)(c * HX + kx) * PY + ky) * n2 + 2 * k;
            X[c] = make_float2(p.zs_x[row[c]], p.zs_x[row[c] + 1]);
        }
        const float2 Y0 = make_float2(kxx * X[0].x + kxy * X[1].x + kxz * X[2].x, kxx * X[0].y + kxy * X[1].y + kxz * X[2].y);
        const float2 Y1 = make_float2(kxy * X[0].x + kyy * X[1].x + kyz * X[2].x, kxy * X[0].y + kyy * X[1].y + kyz * X[2].y);
        const float2 Y2 = make_float2(kxz * X[0].x + kyz * X[1].x + kzz * X[2].x, kxz * X[0].y + kyz * X[1].y + kzz * X[2].y);
        split_store(yhi, ylo, row[0], Y0.x); split_store(yhi, ylo, row[0] + 1, Y0.y);
        split_store(yhi, ylo, row[1], Y1.x); split_store(yhi, ylo, row[1] + 1, Y1.y);
        split_store(yhi, ylo, row[2], Y2.x); split_store(yhi, ylo, row[2] + 1, Y2.y);
    }
}

__global__ void k_zs_scatter(HotParams p, LaunchArgs a) {
    if (a.mode != LM_EVAL && p.st->done) return;
    const long long lines = 3LL * p.hx * p.py;
    const int kp = p.zs_kp, nzp = p.nzp, nz = p.nz;
    if (blockIdx.x == 0 && threadIdx.x == 0 && *p.zs_err) {
        p.st->status = -6;          // MM_ETIMEOUT: a product gave up waiting for its operands
        p.st->done = 1;
    }
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < lines * nz;
         t += (long long)gridDim.x * blockDim.x) {
        const long long l = t / nz;
        const int z = (int)(t % nz);
        p.s2[l * nzp + z] = make_float2(p.zs_o[l * kp + 2 * z], p.zs_o[l * kp + 2 * z + 1]);
    }
}

int grid_of(long long n) {
    const long long g = (n + 255) / 256;
    return (int)(g < 8 * 152 ? (g < 1 ? 1 : g) : 8 * 152);
}

}  // namespace

// sizes[0..6]: A (each of hi, lo), X, Y (each of hi, lo), O, F/G tables (each of 4), error word
size_t zsplit_bytes(int nx, int ny, int nz, int hx, int py, int pz, int nzp, size_t* sizes) {
    (void)nx;
    (void)ny;
    (void)nz;
    const long long lines = 3LL * hx * py;
    const int kp = 2 * nzp, n2 = 2 * pz;
    sizes[0] = a256((size_t)lines * kp * 2);
    sizes[1] = a256((size_t)lines * n2 * 4);
    sizes[2] = a256((size_t)lines * n2 * 2);
    sizes[3] = a256((size_t)lines * kp * 4);
    sizes[4] = a256((size_t)n2 * kp * 2);
    sizes[5] = 256;
    sizes[6] = 0;
    return 2 * sizes[0] + sizes[1] + 2 * sizes[2] + sizes[3] + 4 * sizes[4] + sizes[5];
}

cudaError_t zsplit_tables(const HotParams& p, cudaStream_t s) {
    const int kp = p.zs_kp, n2 = 2 * p.pz;
    cudaError_t e = gemm_configure();
    if (e != cudaSuccess) return e;
    k_zs_tables<<<grid_of((long long)n2 * kp), 256, 0, s>>>(
        p.pz, p.nz, kp, const_cast<bf16*>(static_cast<const bf16*>(p.zs_f_hi)),
        const_cast<bf16*>(static_cast<const bf16*>(p.zs_f_lo)), const_cast<bf16*>(static_cast<const bf16*>(p.zs_g_hi)),
        const_cast<bf16*>(static_cast<const bf16*>(p.zs_g_lo)));
    return cudaGetLastError();
}

cudaError_t launch_zconv_split(const HotParams& p, const LaunchArgs& a, cudaStream_t s) {
    const long long lines = 3LL * p.hx * p.py;
    const int kp = p.zs_kp, n2 = 2 * p.pz;
    cudaError_t e;
    k_zs_gather<<<grid_of(lines * p.nzp), 256, 0, s>>>(p, a);
    if ((e = cudaGetLastError())) return e;
    // X = A_hi F_hi^T + A_hi F_lo^T + A_lo F_hi^T
    if ((e = gemm_bf16(p.zs_a_hi, kp, 0, p.zs_f_hi, kp, 0, p.zs_x, n2, 0, (int)lines, n2, kp, 1, 1.f, 0, p.zs_err, s)))
        return e;
    if ((e = gemm_bf16(p.zs_a_hi, kp, 0, p.zs_f_lo, kp, 0, p.zs_x, n2, 0, (int)lines, n2, kp, 1, 1.f, 1, p.zs_err, s)))
        return e;
    if ((e = gemm_bf16(p.zs_a_lo, kp, 0, p.zs_f_hi, kp, 0, p.zs_x, n2, 0, (int)lines, n2, kp, 1, 1.f, 1, p.zs_err, s)))
        return e;
    k_zs_product<<<grid_of((long long)p.hx * p.py * p.pz), 256, 0, s>>>(p, a);
    if ((e = cudaGetLastError())) return e;
    // O = Y_hi G_hi^T + Y_hi G_lo^T + Y_lo G_hi^T
    if ((e = gemm_bf16(p.zs_y_hi, n2, 0, p.zs_g_hi, n2, 0, p.zs_o, kp, 0, (int)lines, kp, n2, 1, 1.f, 0, p.zs_err, s)))
        return e;
    if ((e = gemm_bf16(p.zs_y_hi, n2, 0, p.zs_g_lo, n2, 0, p.zs_o, kp, 0, (int)lines, kp, n2, 1, 1.f, 1, p.zs_err, s)))
        return e;
    if ((e = gemm_bf16(p.zs_y_lo, n2, 0, p.zs_g_hi, n2, 0, p.zs_o, kp, 0, (int)lines, kp, n2, 1, 1.f, 1, p.zs_err, s)))
        return e;
    k_zs_scatter<<<grid_of(lines * p.nz), 256, 0, s>>>(p, a);
    return cudaGetLastError();
}

}  // namespace mm
