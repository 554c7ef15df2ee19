// fft32.cuh - single-precision complex FFT building blocks for the hot path.
//
// The convolution of Sec. 3.2 (stages i and iii) needs batched 1-D FFTs along
// each axis.  Here each line lives in shared memory; one thread owns one
// radix-16 butterfly per pass (Stockham auto-sort ordering, so input and
// output are both in natural order and no bit reversal is needed).  Values
// stay in registers inside a pass; shared memory carries them between passes.
//
// Shared-memory lines use a padded index pad(i) = i + i/16 so that the
// stride-16 writes of the first pass hit 16 distinct 64-bit bank pairs.
//
// Twiddles come from a table tw[t] = exp(-2 pi i t / TWN) (TWN = 4096)
// computed in double precision on the host and rounded once to float.
#pragma once
#include <cuda_runtime.h>

namespace mmfft {

constexpr int TWN_LOG = 12;
constexpr int TWN = 1 << TWN_LOG;

__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 4) + 1; }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// multiply by -i (forward transform) or +i (inverse transform)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ---- in-register DFTs (sign -1 forward, +1 inverse; no scaling) -------------
template <bool INV>
__device__ __forceinline__ void dft2(float2& a0, float2& a1) {
    float2 t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
    float2 t2 = cadd(a1, a3), t3 = mul_mi<INV>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

// v[0..7] in natural order in, natural order out
template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
    const float c = 0.70710678118654752440f;
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    // o_k *= w8^k
    if (!INV) {
        o1 = make_float2(c * (o1.x + o1.y), c * (o1.y - o1.x));
        o2 = mul_mi<false>(o2);
        o3 = make_float2(c * (o3.y - o3.x), -c * (o3.x + o3.y));
    } else {
        o1 = make_float2(c * (o1.x - o1.y), c * (o1.x + o1.y));
        o2 = mul_mi<true>(o2);
        o3 = make_float2(-c * (o3.x + o3.y), c * (o3.x - o3.y));
    }
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
    // cos/sin of k*pi/8, k = 1..7
    const float C1 = 0.92387953251128675613f, S1 = 0.38268343236508977173f;
    const float C2 = 0.70710678118654752440f;
    float2 e[8], o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) { e[k] = v[2 * k]; o[k] = v[2 * k + 1]; }
    dft8<INV>(e);
    dft8<INV>(o);
    const float cs[8] = {1.f, C1, C2, S1, 0.f, -S1, -C2, -C1};
    const float sn[8] = {0.f, S1, C2, C1, 1.f, C1, C2, S1};
#pragma unroll
    for (int k = 1; k < 8; ++k) {
        float2 w = make_float2(cs[k], INV ? sn[k] : -sn[k]);
        o[k] = cmul(o[k], w);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        v[k] = cadd(e[k], o[k]);
        v[k + 8] = csub(e[k], o[k]);
    }
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        dft2<INV>(v[0], v[1]);
    } else if constexpr (R == 4) {
        dft4<INV>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 8) {
        dft8<INV>(v);
    } else {
        static_assert(R == 16, "radix");
        dft16<INV>(v);
    }
}

// twiddle W^{k r}, W = exp(-+2 pi i /(Ns R)), read from the TWN table
template <bool INV>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int t) {
    float2 w = __ldg(tw + t);
    return INV ? cconj(w) : w;
}

// Main radix of a line of length 2^LOGP and the number of radix-16 passes.
template <int LOGP>
struct Plan {
    static constexpr int P = 1 << LOGP;
    static constexpr int R = LOGP >= 4 ? 16 : P;        // registers per thread
    static constexpr int NB = P / R;                    // threads per line
    static constexpr int N16 = LOGP >= 4 ? LOGP / 4 : 0;
    static constexpr int REM = LOGP >= 4 ? (1 << (LOGP % 4)) : 1;   // trailing radix
};

// In-place FFT of `nlines` lines of length 2^LOGP stored in shared memory at
// line l -> base + l*lstride (padded indices).  Threads [0, nlines*NB) work;
// the rest only join the barriers.  Must be called by every thread of the
// block.  Direction INV (no 1/P scaling).
template <int LOGP, bool INV>
__device__ void fft_lines(float2* base, int nlines, int lstride, const float2* __restrict__ tw) {
    using PL = Plan<LOGP>;
    constexpr int P = PL::P, R = PL::R, NB = PL::NB;
    const int tid = threadIdx.x;
    const bool active = tid < nlines * NB;
    const int line = active ? tid / NB : 0;
    const int j = active ? tid - line * NB : 0;
    float2* a = base + line * lstride;
    float2 v[R];

    if constexpr (LOGP == 0) {
        __syncthreads();
    } else if constexpr (LOGP < 4) {
        // single pass of radix P, Ns = 1 (no twiddles)
        if (active) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = a[pad(r)];
            dft<R, INV>(v);
#pragma unroll
            for (int r = 0; r < R; ++r) a[pad(r)] = v[r];
        }
        __syncthreads();
    } else {
        int Ns = 1;
#pragma unroll 1
        for (int p = 0; p < PL::N16; ++p) {
            if (active) {
#pragma unroll
                for (int r = 0; r < 16; ++r) v[r] = a[pad(j + r * NB)];
                const int k = j & (Ns - 1);
                if (Ns > 1) {
                    const int step = k * (TWN / (Ns * 16));
#pragma unroll
                    for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], twiddle<INV>(tw, r * step));
                }
                dft<16, INV>(v);
            }
            __syncthreads();
            if (active) {
                const int k = j & (Ns - 1);
                const int o = (j - k) * 16 + k;
#pragma unroll
                for (int r = 0; r < 16; ++r) a[pad(o + r * Ns)] = v[r];
            }
            __syncthreads();
            Ns *= 16;
        }
        if constexpr (PL::REM > 1) {
            constexpr int RR = PL::REM;          // 2, 4 or 8
            constexpr int NBR = P / RR;          // butterflies of radix RR per line
            constexpr int PER = 16 / RR;         // per thread
            if (active) {
#pragma unroll
                for (int b = 0; b < PER; ++b) {
                    const int jj = j + b * NB;
#pragma unroll
                    for (int r = 0; r < RR; ++r) v[b * RR + r] = a[pad(jj + r * NBR)];
                }
#pragma unroll
                for (int b = 0; b < PER; ++b) {
                    const int jj = j + b * NB;
                    const int k = jj & (Ns - 1);
                    const int step = k * (TWN / (Ns * RR));
#pragma unroll
                    for (int r = 1; r < RR; ++r) v[b * RR + r] = cmul(v[b * RR + r], twiddle<INV>(tw, r * step));
                    dft<RR, INV>(v + b * RR);
                }
            }
            __syncthreads();
            if (active) {
#pragma unroll
                for (int b = 0; b < PER; ++b) {
                    const int jj = j + b * NB;
                    const int k = jj & (Ns - 1);
                    const int o = (jj - k) * RR + k;
#pragma unroll
                    for (int r = 0; r < RR; ++r) a[pad(o + r * Ns)] = v[b * RR + r];
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace mmfft
