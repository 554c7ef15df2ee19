// setup.cu - the demagnetising kernel, built once per geometry in FP64.
//
// Sec. 2.1.1 (Eq. 2): the magnetostatic field is a convolution of M with
// grad grad (1/r); on a grid of identical cuboids the convolution weights are
// the cell-averaged tensor N_ab(offset) (closed form by Newell, Williams &
// Dunlop 1993; the paper does not name its formula).  Sec. 3.2: the kernel is
// kept fully symmetric so its transform is real, which halves its storage and
// makes the point-wise product real-times-complex.
//
// Steps (all on the GPU, FP64 except the final store):
//  1. k_tensor_octant - N_ab on the non-negative offsets (the other octants
//     follow from parity: diagonal components even, N_xy odd in x and y,
//     ...).  Near the origin Newell's closed form; further out its 27-term
//     sum cancels catastrophically, so the same cell average is integrated
//     numerically: for separated cells it is (1/V) Int D(r + w) T(w) dw with
//     D the point-dipole kernel and T the box-overlap tent, done with
//     Gauss-Legendre nodes on each half of every axis.  Periodic axes
//     (Sec. 2.1.1) sum 2P+1 images (2P+2 for the mirror-symmetric offset n/2).
//  2. k_wrap - one component on the padded grid (wrap-around layout).
//  3. k_fft64_axis - FP64 complex FFT along x, y, z (radix-2 Stockham).
//  4. k_store_octant - real part times -1/(Px Py Pz) to float32 on the
//     kx, ky, kz >= 0 octant; the largest |Im| is recorded as a check.
#include "mm_internal.cuh"
#include <math.h>

namespace mm {

__device__ __forceinline__ double sq(double v) { return v * v; }

// Newell's f; symmetric in y <-> z
__device__ double newell_f(double x, double y, double z) {
    const double x2 = x * x, y2 = y * y, z2 = z * z;
    const double R = sqrt(x2 + y2 + z2);
    double acc = (2.0 * x2 - y2 - z2) * R * (1.0 / 6.0);
    double c = 0.5 * y * (z2 - x2);
    if (c != 0.0) acc += c * asinh(y / sqrt(x2 + z2));
    c = 0.5 * z * (y2 - x2);
    if (c != 0.0) acc += c * asinh(z / sqrt(x2 + y2));
    c = x * y * z;
    if (c != 0.0) acc -= c * atan(y * z / (x * R));
    return acc;
}

// Newell's g (for the off-diagonal components)
__device__ double newell_g(double x, double y, double z) {
    const double x2 = x * x, y2 = y * y, z2 = z * z;
    const double R = sqrt(x2 + y2 + z2);
    double acc = -x * y * R * (1.0 / 3.0);
    double c = x * y * z;
    if (c != 0.0) acc += c * asinh(z / sqrt(x2 + y2));
    c = y * (3.0 * z2 - y2) * (1.0 / 6.0);
    if (c != 0.0) acc += c * asinh(x / sqrt(y2 + z2));
    c = x * (3.0 * z2 - x2) * (1.0 / 6.0);
    if (c != 0.0) acc += c * asinh(y / sqrt(x2 + z2));
    c = z * z2 * (1.0 / 6.0);
    if (c != 0.0) acc -= c * atan(x * y / (z * R));
    c = 0.5 * z * y2;
    if (c != 0.0) acc -= c * atan(x * z / (y * R));
    c = 0.5 * z * x2;
    if (c != 0.0) acc -= c * atan(y * z / (x * R));
    return acc;
}

// 27-point second difference with weights (-1, 2, -1) per axis, / (4 pi V)
template <bool G>
__device__ double newell_sum(double a, double b, double c, double da, double db, double dc) {
    double acc = 0.0;
    for (int i = -1; i <= 1; ++i) {
        const double wi = i == 0 ? 2.0 : -1.0;
        for (int j = -1; j <= 1; ++j) {
            const double wj = j == 0 ? 2.0 : -1.0;
            for (int k = -1; k <= 1; ++k) {
                const double wk = k == 0 ? 2.0 : -1.0;
                const double fa = a + i * da, fb = b + j * db, fc = c + k * dc;
                acc += wi * wj * wk * (G ? newell_g(fa, fb, fc) : newell_f(fa, fb, fc));
            }
        }
    }
    return acc / (4.0 * M_PI * da * db * dc);
}

// out: xx yy zz xy xz yz
__device__ void tensor_newell(double X, double Y, double Z, double dx, double dy, double dz, double* out) {
    out[0] = newell_sum<false>(X, Y, Z, dx, dy, dz);
    out[1] = newell_sum<false>(Y, X, Z, dy, dx, dz);
    out[2] = newell_sum<false>(Z, Y, X, dz, dy, dx);
    out[3] = newell_sum<true>(X, Y, Z, dx, dy, dz);
    out[4] = newell_sum<true>(X, Z, Y, dx, dz, dy);
    out[5] = newell_sum<true>(Y, Z, X, dy, dz, dx);
}

__device__ void tensor_quadrature(double X, double Y, double Z, const SetupParams& p, int q, double* out) {
    const int n = p.gl_n[q];
    const double V = p.dx * p.dy * p.dz;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    // 2n nodes per axis: w = +-d (t+1)/2, weight d/2 * w_gl * (d - |w|)
    for (int a = 0; a < 2 * n; ++a) {
        const int ia = a < n ? a : a - n;
        const double wa0 = 0.5 * p.dx * (p.gl_t[q][ia] + 1.0);
        const double wa = a < n ? wa0 : -wa0;
        const double ga = 0.5 * p.dx * p.gl_w[q][ia] * (p.dx - wa0);
        const double sx = X + wa;
        for (int b = 0; b < 2 * n; ++b) {
            const int ib = b < n ? b : b - n;
            const double wb0 = 0.5 * p.dy * (p.gl_t[q][ib] + 1.0);
            const double wb = b < n ? wb0 : -wb0;
            const double gb = 0.5 * p.dy * p.gl_w[q][ib] * (p.dy - wb0);
            const double sy = Y + wb;
            for (int c = 0; c < 2 * n; ++c) {
                const int ic = c < n ? c : c - n;
                const double wc0 = 0.5 * p.dz * (p.gl_t[q][ic] + 1.0);
                const double wc = c < n ? wc0 : -wc0;
                const double gc = 0.5 * p.dz * p.gl_w[q][ic] * (p.dz - wc0);
                const double sz = Z + wc;
                const double r2 = sx * sx + sy * sy + sz * sz;
                const double inv5 = 1.0 / (r2 * r2 * sqrt(r2));
                const double w = -ga * gb * gc * inv5;      // 1/(4 pi V) applied at the end
                acc[0] += w * (3.0 * sx * sx - r2);
                acc[1] += w * (3.0 * sy * sy - r2);
                acc[2] += w * (3.0 * sz * sz - r2);
                acc[3] += w * 3.0 * sx * sy;
                acc[4] += w * 3.0 * sx * sz;
                acc[5] += w * 3.0 * sy * sz;
            }
        }
    }
    const double s = 1.0 / (4.0 * M_PI * V);
    for (int i = 0; i < 6; ++i) out[i] = acc[i] * s;
}

// cell-averaged tensor at physical offset (lengths scaled so the largest
// cell edge is 1): closed form below 4 edges, quadrature beyond, with the
// node count graded by distance (the float64 closed form loses ~dist^5 ulps;
// the quadrature converges like (4 dist)^(-2n))
__device__ void tensor_at(double X, double Y, double Z, const SetupParams& p, double* out) {
    const double dist = sqrt(X * X + Y * Y + Z * Z);
    if (dist < 4.0) {
        tensor_newell(X, Y, Z, p.dx, p.dy, p.dz, out);
        return;
    }
    const int q = dist < 10.0 ? 3 : dist < 25.0 ? 2 : dist < 80.0 ? 1 : 0;
    tensor_quadrature(X, Y, Z, p, q, out);
}

__device__ __forceinline__ void image_range(int o, int n, bool periodic, int P, int& lo, int& hi) {
    if (!periodic) { lo = hi = 0; return; }
    lo = -P; hi = P;
    if ((n & 1) == 0 && 2 * o == n) lo = -P - 1;      // mirror-symmetric image set
}

__global__ void k_tensor_octant(SetupParams p) {
    const long long total = (long long)p.ox * p.oy * p.oz;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int ox = (int)(idx % p.ox);
        const int oy = (int)((idx / p.ox) % p.oy);
        const int oz = (int)(idx / ((long long)p.ox * p.oy));
        int lx, hx, ly, hy, lz, hz;
        image_range(ox, p.nx, p.pbc[0], p.images, lx, hx);
        image_range(oy, p.ny, p.pbc[1], p.images, ly, hy);
        image_range(oz, p.nz, p.pbc[2], p.images, lz, hz);
        double sum[6] = {0, 0, 0, 0, 0, 0}, t[6];
        for (int iz = lz; iz <= hz; ++iz)
            for (int iy = ly; iy <= hy; ++iy)
                for (int ix = lx; ix <= hx; ++ix) {
                    const double X = (double)(ox + ix * p.nx) * p.dx;
                    const double Y = (double)(oy + iy * p.ny) * p.dy;
                    const double Z = (double)(oz + iz * p.nz) * p.dz;
                    tensor_at(X, Y, Z, p, t);
                    for (int c = 0; c < 6; ++c) sum[c] += t[c];
                }
        for (int c = 0; c < 6; ++c) p.oct[c * total + idx] = sum[c];
    }
}

// padded index -> octant index and whether it mirrors a negative offset
__device__ __forceinline__ bool axis_map(int i, int n, int P, bool periodic, int& o, bool& neg) {
    if (periodic) {
        if (2 * i <= n) { o = i; neg = false; } else { o = n - i; neg = true; }
        return true;
    }
    if (i < n) { o = i; neg = false; return true; }
    if (i > P - n) { o = P - i; neg = true; return true; }
    return false;
}

__global__ void k_wrap(SetupParams p, int comp) {
    const long long total = (long long)p.px * p.py * p.pz;
    const long long otot = (long long)p.ox * p.oy * p.oz;
    // odd axes of each component: xx yy zz xy xz yz
    const int oddx = comp == 3 || comp == 4, oddy = comp == 3 || comp == 5, oddz = comp == 4 || comp == 5;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % p.px);
        const int j = (int)((idx / p.px) % p.py);
        const int k = (int)(idx / ((long long)p.px * p.py));
        int ox, oy, oz;
        bool nx_, ny_, nz_;
        double v = 0.0;
        if (axis_map(i, p.nx, p.px, p.pbc[0], ox, nx_) && axis_map(j, p.ny, p.py, p.pbc[1], oy, ny_) &&
            axis_map(k, p.nz, p.pz, p.pbc[2], oz, nz_)) {
            v = p.oct[comp * otot + ((long long)oz * p.oy + oy) * p.ox + ox];
            if ((oddx && nx_) ^ (oddy && ny_) ^ (oddz && nz_)) v = -v;
        }
        p.work[idx] = make_double2(v, 0.0);
    }
}

// FP64 Stockham FFT (forward) of one line of L = r0 * 2^logL points per block
// in shared memory: for an odd factor r0 (3, 5, 7) a first pass of radix r0
// (a direct r0-point DFT, out of place into the second half of the shared
// buffer and back), then radix-2 passes.  Line q starts at
// (q % ninner) * sinner + (q / ninner) * souter; elements es apart.
__global__ void k_fft64_axis(double2* data, int logL, int r0, long long es, int ninner, long long sinner,
                             long long souter) {
    extern __shared__ double2 sd[];
    const int L = r0 << logL;
    const long long q = blockIdx.x;
    double2* line = data + (q % ninner) * sinner + (q / ninner) * souter;
    for (int i = threadIdx.x; i < L; i += blockDim.x) sd[i] = line[i * es];
    __syncthreads();
    int ns0 = 1;
    if (r0 > 1) {
        // radix r0, Ns = 1: inputs b + r Q, outputs b r0 + k
        const int Q = L / r0;
        double2* sd2 = sd + L;
        for (int b = threadIdx.x; b < Q; b += blockDim.x) {
            for (int k = 0; k < r0; ++k) {
                double2 acc = make_double2(0.0, 0.0);
                for (int r = 0; r < r0; ++r) {
                    double sn, cs;
                    sincospi(-2.0 * (double)((r * k) % r0) / (double)r0, &sn, &cs);
                    const double2 x = sd[b + r * Q];
                    acc.x += x.x * cs - x.y * sn;
                    acc.y += x.x * sn + x.y * cs;
                }
                sd2[b * r0 + k] = acc;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < L; i += blockDim.x) sd[i] = sd2[i];
        __syncthreads();
        ns0 = r0;
    }
    const int half = L >> 1;
    for (int Ns = ns0; Ns < L; Ns <<= 1) {
        double2 r0v[8], r1v[8];
        int cnt = 0;
        for (int jb = threadIdx.x; jb < half; jb += blockDim.x, ++cnt) {
            const int k = jb % Ns;
            const double2 a0 = sd[jb], a1 = sd[jb + half];
            double s, c;
            sincospi(-(double)k / (double)Ns, &s, &c);
            const double2 b = make_double2(a1.x * c - a1.y * s, a1.x * s + a1.y * c);
            r0v[cnt] = make_double2(a0.x + b.x, a0.y + b.y);
            r1v[cnt] = make_double2(a0.x - b.x, a0.y - b.y);
        }
        __syncthreads();
        cnt = 0;
        for (int jb = threadIdx.x; jb < half; jb += blockDim.x, ++cnt) {
            const int k = jb % Ns;
            const int o = (jb - k) * 2 + k;
            sd[o] = r0v[cnt];
            sd[o + Ns] = r1v[cnt];
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < L; i += blockDim.x) line[i * es] = sd[i];
}

__global__ void k_store_octant(SetupParams p, int comp, double scale) {
    const long long total = (long long)p.hx * p.hyk * p.hzk;
    double mre = 0.0, mim = 0.0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int kz = (int)(idx % p.hzk);
        const int ky = (int)((idx / p.hzk) % p.hyk);
        const int kx = (int)(idx / ((long long)p.hzk * p.hyk));
        const double2 v = p.work[((long long)kz * p.py + ky) * p.px + kx];
        p.kt[comp * total + idx] = (float)(v.x * scale);
        mre = fmax(mre, fabs(v.x));
        mim = fmax(mim, fabs(v.y));
    }
    atomicMax(&p.st->kre_bits, (unsigned long long)__double_as_longlong(mre));
    atomicMax(&p.st->kim_bits, (unsigned long long)__double_as_longlong(mim));
}

cudaError_t launch_kernel_setup(const SetupParams& p, cudaStream_t s) {
    const long long otot = (long long)p.ox * p.oy * p.oz;
    int blocks = (int)((otot + 127) / 128);
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_tensor_octant<<<blocks, 128, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    const long long ptot = (long long)p.px * p.py * p.pz;
    const double scale = -1.0 / (double)ptot;
    // each length is r * 2^l with an odd factor r (1, 3, 5 or 7)
    auto split = [](int n, int& l, int& r) {
        l = 0;
        while (((n >> l) & 1) == 0 && (1 << l) < n) ++l;
        r = n >> l;
    };
    int lx, ly, lz, rx, ry, rz;
    split(p.px, lx, rx);
    split(p.py, ly, ry);
    split(p.pz, lz, rz);
    // the odd-radix pass works out of place: twice the line in shared memory
    auto smem = [](int n, int r) { return (size_t)(r > 1 ? 2 : 1) * n * sizeof(double2); };
    const size_t sm_max = 2 * 4096 * sizeof(double2);
    if ((e = cudaFuncSetAttribute(k_fft64_axis, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_max))) return e;
    for (int comp = 0; comp < p.ncomp; ++comp) {
        int wb = (int)((ptot + 255) / 256);
        if (wb > 152 * 32) wb = 152 * 32;
        k_wrap<<<wb, 256, 0, s>>>(p, comp);
        // x lines: contiguous, one per (y, z)
        if (p.px > 1)
            k_fft64_axis<<<p.py * p.pz, p.px / 2 < 512 ? (p.px / 2 < 32 ? 32 : p.px / 2) : 512,
                           smem(p.px, rx), s>>>(p.work, lx, rx, 1, 1, p.px, p.px);
        // y lines: stride px, one per (x, z)
        if (p.py > 1)
            k_fft64_axis<<<p.px * p.pz, p.py / 2 < 512 ? (p.py / 2 < 32 ? 32 : p.py / 2) : 512,
                           smem(p.py, ry), s>>>(p.work, ly, ry, p.px, p.px, 1, (long long)p.px * p.py);
        // z lines: stride px*py, one per (x, y)
        if (p.pz > 1)
            k_fft64_axis<<<p.px * p.py, p.pz / 2 < 512 ? (p.pz / 2 < 32 ? 32 : p.pz / 2) : 512,
                           smem(p.pz, rz), s>>>(p.work, lz, rz, (long long)p.px * p.py, p.px * p.py, 1, 0);
        int sb = (int)(((long long)p.hx * p.hyk * p.hzk + 255) / 256);
        if (sb > 152 * 32) sb = 152 * 32;
        k_store_octant<<<sb, 256, 0, s>>>(p, comp, scale);
        if ((e = cudaGetLastError())) return e;
    }
    return cudaSuccess;
}

}  // namespace mm
