// hotpath_yz.cu - the y and z stages of the convolution of Sec. 3.2 in ONE pass
// for 3-D grids with few z cells (nz <= 8, the thin samples of an ensemble).
//
// The general 3-D path runs a y forward pass (writing the z-padded spectrum
// s2), the z column pass with the kernel product, and a y inverse pass: three
// round trips through HBM of a spectrum Pz/nz times larger than the x
// spectrum.  Here one block owns one kx column of the x spectrum s1
// [c][kx][z][y] for every z < nz: it transforms the 3 nz lines along y in
// shared memory, then one thread per ky transforms the z line of each
// component (nz inputs zero-padded to Pz: a register FFT; a direct DFT for a
// periodic z axis, Pz = nz), multiplies
// by the real symmetric kernel at every (ky, kz) (Sec. 3.2 stage ii; xy and
// yz odd in ky, xz and yz odd in kz) and transforms back to the nz outputs it
// needs, and the block finishes with the inverse y transforms.  An evaluation
// of such a grid is then three passes, like a 2-D one.
#include "hotpath_kernels.cuh"

namespace mm {

namespace {

// NZ: the z cells the block's registers hold (2, 3, 4 or 8; nz <= NZ)
template <int LOGP, int NZ>
struct YZ {
    static constexpr int P = 1 << LOGP;
    static constexpr int NL = 3 * NZ;                       // lines (component, z) of P points
    static constexpr int NT = mmfft::threads_of(NL, LOGP);
    static constexpr int LS = mmfft::padded_len(P);
    static constexpr int PZC = NZ == 3 ? 8 : 2 * NZ;        // Pz of an open z axis of NZ cells
    static constexpr size_t SMEM = (size_t)(NL * LS + PZC) * sizeof(float2);
    // resident blocks asked of the register allocator: the blocks are many
    // (one per kx column of every sample) and each waits on its loads, so
    // residency matters more than a few spilled values (nz <= 8 keeps 48
    // complex values per thread in the z stage and one block)
    static constexpr int MINB = NZ == 8 ? 1 : (NT >= 512 ? 1 : (1024 / NT > 4 ? 4 : 1024 / NT));
};

template <int LOGP, int NZ>
__device__ __forceinline__ void yzconv_body(const HotParams& p, const LaunchArgs& a, int kx) {
    using namespace mmfft;
    using S = YZ<LOGP, NZ>;
    extern __shared__ float2 sm[];
    float2* tz = sm + S::NL * S::LS;                        // exp(-2 pi i t / Pz), t < Pz
    const int nz = p.nz, PZ = p.pz, NY = p.ny, HX = p.hx;
    const long long nyp = p.nyp;
    // the block's lines: l = c NZ + z, y < ny from s1, zero elsewhere; every
    // load of the thread in flight before the first store, and before the
    // run-state check (a finished run returns before anything is written)
    {
        const bool done = a.mode != LM_EVAL && p.st->done;
        constexpr int IT = (S::NL * S::P + S::NT - 1) / S::NT;
        float2 v[IT];
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const int idx = threadIdx.x + it * S::NT;
            const int l = idx >> LOGP, y = idx & (S::P - 1);
            const int c = l / NZ, z = l - c * NZ;
            v[it] = make_float2(0.f, 0.f);
            if (idx < S::NL * S::P && z < nz && y < NY) v[it] = p.s1[((long long)(c * HX + kx) * nz + z) * nyp + y];
        }
        if (done) return;
        for (int t = threadIdx.x; t < PZ; t += S::NT) tz[t] = p.tw[t * (TWN / PZ)];
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const int idx = threadIdx.x + it * S::NT;
            if (idx < S::NL * S::P) sm[(idx >> LOGP) * S::LS + pad(idx & (S::P - 1))] = v[it];
        }
    }
    __syncthreads();
    fft_lines<LOGP, S::NL, false>(sm, p.tw);
    // z: one thread per ky, the three components' z lines in registers
    const long long cs = (long long)HX * p.hyk * p.hzk;
    for (int ky = threadIdx.x; ky < S::P; ky += S::NT) {
        const bool yh = ky > (S::P >> 1);
        const int kyq = yh ? S::P - ky : ky;
        const float* kb = p.kt + ((long long)kx * p.hyk + kyq) * p.hzk;
        if (PZ == S::PZC) {
            // open z: register FFTs of the Pz-point lines (zero past nz)
            constexpr int PZC = S::PZC;
            float2 X[3][PZC];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
#pragma unroll
                for (int z = 0; z < PZC; ++z)
                    X[c][z] = z < NZ ? sm[(c * NZ + z) * S::LS + pad(ky)] : make_float2(0.f, 0.f);
                dft<PZC, false>(X[c]);
            }
#pragma unroll
            for (int kz = 0; kz < PZC; ++kz) {
                constexpr int H = PZC / 2;
                const bool hi = kz > H;
                const int kzq = hi ? PZC - kz : kz;
                const float kxx = __ldg(kb + kzq), kyy = __ldg(kb + cs + kzq), kzz = __ldg(kb + 2 * cs + kzq);
                float kxy = __ldg(kb + 3 * cs + kzq), kxz = __ldg(kb + 4 * cs + kzq), kyz = __ldg(kb + 5 * cs + kzq);
                if (yh) { kxy = -kxy; kyz = -kyz; }
                if (hi) { kxz = -kxz; kyz = -kyz; }
                const float2 A = X[0][kz], Bv = X[1][kz], C = X[2][kz];
                X[0][kz] = make_float2(kxx * A.x + kxy * Bv.x + kxz * C.x, kxx * A.y + kxy * Bv.y + kxz * C.y);
                X[1][kz] = make_float2(kxy * A.x + kyy * Bv.x + kyz * C.x, kxy * A.y + kyy * Bv.y + kyz * C.y);
                X[2][kz] = make_float2(kxz * A.x + kyz * Bv.x + kzz * C.x, kxz * A.y + kyz * Bv.y + kzz * C.y);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dft<PZC, true>(X[c]);
#pragma unroll
                for (int z = 0; z < NZ; ++z) sm[(c * NZ + z) * S::LS + pad(ky)] = X[c][z];
            }
            continue;
        }
        // periodic z (Pz = nz <= NZ): the direct DFT of the Pz-point lines
        float2 av[3][NZ], out[3][NZ];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int z = 0; z < NZ; ++z) {
                av[c][z] = sm[(c * NZ + z) * S::LS + pad(ky)];
                out[c][z] = make_float2(0.f, 0.f);
            }
        for (int kz = 0; kz < PZ; ++kz) {
            const bool hi = kz > (PZ >> 1);
            const int kzq = hi ? PZ - kz : kz;
            const float kxx = __ldg(kb + kzq), kyy = __ldg(kb + cs + kzq), kzz = __ldg(kb + 2 * cs + kzq);
            float kxy = __ldg(kb + 3 * cs + kzq), kxz = __ldg(kb + 4 * cs + kzq), kyz = __ldg(kb + 5 * cs + kzq);
            if (yh) { kxy = -kxy; kyz = -kyz; }
            if (hi) { kxz = -kxz; kyz = -kyz; }
            float2 Xv[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
            for (int z = 0; z < NZ; ++z) {
                const float2 w = tz[(z * kz) & (PZ - 1)];
#pragma unroll
                for (int c = 0; c < 3; ++c) Xv[c] = cadd(Xv[c], cmul(av[c][z], w));
            }
            const float2 Y0 = make_float2(kxx * Xv[0].x + kxy * Xv[1].x + kxz * Xv[2].x,
                                          kxx * Xv[0].y + kxy * Xv[1].y + kxz * Xv[2].y);
            const float2 Y1 = make_float2(kxy * Xv[0].x + kyy * Xv[1].x + kyz * Xv[2].x,
                                          kxy * Xv[0].y + kyy * Xv[1].y + kyz * Xv[2].y);
            const float2 Y2 = make_float2(kxz * Xv[0].x + kyz * Xv[1].x + kzz * Xv[2].x,
                                          kxz * Xv[0].y + kyz * Xv[1].y + kzz * Xv[2].y);
#pragma unroll
            for (int z = 0; z < NZ; ++z) {
                const float2 w = cconj(tz[(z * kz) & (PZ - 1)]);
                out[0][z] = cadd(out[0][z], cmul(Y0, w));
                out[1][z] = cadd(out[1][z], cmul(Y1, w));
                out[2][z] = cadd(out[2][z], cmul(Y2, w));
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int z = 0; z < NZ; ++z) sm[(c * NZ + z) * S::LS + pad(ky)] = out[c][z];
    }
    __syncthreads();
    fft_lines<LOGP, S::NL, true>(sm, p.tw);
    for (int idx = threadIdx.x; idx < S::NL * S::P; idx += S::NT) {
        const int l = idx >> LOGP, y = idx & (S::P - 1);
        const int c = l / NZ, z = l - c * NZ;
        if (z < nz && y < NY) p.s1[((long long)(c * HX + kx) * nz + z) * nyp + y] = sm[l * S::LS + pad(y)];
    }
}

template <int LOGP, int NZ>
__global__ void __launch_bounds__(YZ<LOGP, NZ>::NT, YZ<LOGP, NZ>::MINB) k_yzconv(HotParams p, LaunchArgs a) {
    yzconv_body<LOGP, NZ>(p, a, blockIdx.x);
}
template <int LOGP, int NZ>
__global__ void __launch_bounds__(YZ<LOGP, NZ>::NT, YZ<LOGP, NZ>::MINB)
kb_yzconv(const HotParams* __restrict__ ps, const int4* __restrict__ work, LaunchArgs a) {
    const int4 w = work[blockIdx.x];
    __shared__ HotParams s_hp;
    load_params(ps + w.x, &s_hp);
    yzconv_body<LOGP, NZ>(s_hp, a, w.y);
}

// y lengths 2^3 .. 2^10 with nz = 2, 3, 4, 2^3 .. 2^8 with nz = 5 .. 8 (the
// lines fit the shared memory of a block; at 2^9 points and 8 z cells the 768
// threads' register budget spills the z stage's 48 complex values per thread)
#define MM_YZ_SHAPES(X) X(3, 2) X(4, 2) X(5, 2) X(6, 2) X(7, 2) X(8, 2) X(9, 2) X(10, 2) \
    X(3, 3) X(4, 3) X(5, 3) X(6, 3) X(7, 3) X(8, 3) X(9, 3) X(10, 3) \
    X(3, 4) X(4, 4) X(5, 4) X(6, 4) X(7, 4) X(8, 4) X(9, 4) X(10, 4) \
    X(3, 8) X(4, 8) X(5, 8) X(6, 8) X(7, 8) X(8, 8)

}  // namespace

// 2, 3, 4 or 8: the fused pass applies with that many z cells per block; 0: it does not
int yz_fused_nz(const HotParams& p) {
    if (p.nz < 2 || p.nz > 8 || p.ry != 1 || p.rz != 1 || p.zsplit) return 0;
    const int nzc = p.nz <= 4 ? p.nz : 8;
    switch (p.logpy * 100 + nzc) {
#define MM_CASE(L, N) case L * 100 + N: return N;
        MM_YZ_SHAPES(MM_CASE)
#undef MM_CASE
        default: return 0;
    }
}

cudaError_t launch_yzconv(const HotParams& p, const LaunchArgs& a, cudaStream_t s) {
    switch (p.logpy * 100 + yz_fused_nz(p)) {
#define MM_CASE(L, N) \
    case L * 100 + N: k_yzconv<L, N><<<p.hx, YZ<L, N>::NT, YZ<L, N>::SMEM, s>>>(p, a); break;
        MM_YZ_SHAPES(MM_CASE)
#undef MM_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// code = logpy * 100 + NZ (the batch groups samples by it)
cudaError_t launch_yzconv_batched(const HotParams* ps, const int4* work, int nb, const LaunchArgs& a, int code,
                                  cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    switch (code) {
#define MM_CASE(L, N) \
    case L * 100 + N: kb_yzconv<L, N><<<nb, YZ<L, N>::NT, YZ<L, N>::SMEM, s>>>(ps, work, a); break;
        MM_YZ_SHAPES(MM_CASE)
#undef MM_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t configure_yz_kernels() {
    cudaError_t e = cudaSuccess;
#define MM_SET(L, N)                                                                                         \
    if ((e = cudaFuncSetAttribute(k_yzconv<L, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024))) \
        return e;                                                                                            \
    if ((e = cudaFuncSetAttribute(kb_yzconv<L, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024))) \
        return e;
    MM_YZ_SHAPES(MM_SET)
#undef MM_SET
    return e;
}

}  // namespace mm
