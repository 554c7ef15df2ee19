// fft32.cuh - single-precision complex FFT building blocks for the hot path.
//
// The convolution of Sec. 3.2 (stages i and iii) needs batched 1-D FFTs along
// each axis.  Each line lives in shared memory; one thread owns one radix-16
// butterfly per pass (Stockham auto-sort ordering: natural order in and out,
// no bit reversal).  Values stay in registers inside a pass; shared memory
// carries them between passes.
//
// Shared-memory lines use a padded index pad(i) = i + i/16 so that the
// stride-16 writes of the first pass hit 16 distinct 64-bit bank pairs.
//
// Twiddles: a table tw[t] = exp(-2 pi i t / TWN) (TWN = 4096) computed in
// double precision on the host and rounded once.  A radix-16 butterfly reads
// only w, w^2, w^4, w^8 and forms the other eleven powers by at most three
// complex products, which keeps the loads off the critical path.
//
// Line counts and lengths are template parameters so that every index is a
// shift or a mask.
#pragma once
#include <cuda_runtime.h>

namespace mmfft {

constexpr int TWN_LOG = 12;
constexpr int TWN = 1 << TWN_LOG;

__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 4) + 1; }

// ---- launch shapes, shared with the host ----------------------------------
// threads per line (one radix-16 butterfly each)
__host__ __device__ constexpr int nb_of(int logp) { return logp >= 4 ? (1 << (logp - 4)) : 1; }
// rows (per component) handled by one block of the x passes: 3*TY/2 complex lines
__host__ __device__ constexpr int ty_of(int logp) {
    return 24 * nb_of(logp) <= 512 ? 16 : 12 * nb_of(logp) <= 512 ? 8 : 6 * nb_of(logp) <= 512 ? 4 : 2;
}
// lines of each component per block for the column passes (3 components each)
__host__ __device__ constexpr int cols_of(int logp, int cap) {
    return (3 * 64 * nb_of(logp) <= 512 && cap >= 64) ? 64
         : (3 * 32 * nb_of(logp) <= 512 && cap >= 32) ? 32
         : (3 * 16 * nb_of(logp) <= 512 && cap >= 16) ? 16
         : (3 * 8 * nb_of(logp) <= 512 && cap >= 8) ? 8
         : (3 * 4 * nb_of(logp) <= 512 && cap >= 4) ? 4
         : (3 * 2 * nb_of(logp) <= 512 && cap >= 2) ? 2 : 1;
}
__host__ __device__ constexpr int tz_of(int logp) { return cols_of(logp, 8); }     // 3-D y passes
// the same tile rules for lines of any length P = r * 2^a (P/16 threads per line)
__host__ __device__ constexpr int cols_of_len(int P, int cap) {
    return (3 * 64 * (P / 16) <= 512 && cap >= 64) ? 64
         : (3 * 32 * (P / 16) <= 512 && cap >= 32) ? 32
         : (3 * 16 * (P / 16) <= 512 && cap >= 16) ? 16
         : (3 * 8 * (P / 16) <= 512 && cap >= 8) ? 8
         : (3 * 4 * (P / 16) <= 512 && cap >= 4) ? 4
         : (3 * 2 * (P / 16) <= 512 && cap >= 2) ? 2 : 1;
}
__host__ __device__ constexpr int tz_of_len(int P) { return cols_of_len(P, 8); }
__host__ __device__ constexpr int threads_of(int nlines, int logp) {
    return ((nlines * nb_of(logp) + 31) / 32) * 32 < 64 ? 64 : ((nlines * nb_of(logp) + 31) / 32) * 32;
}

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

template <bool INV>
__device__ __forceinline__ float2 ldtw(const float2* __restrict__ tw, int t) {
    float2 w = __ldg(tw + t);
    return INV ? cconj(w) : w;
}

// v[r] *= w^r for r = 1..R-1, w = tw[t1] (conjugated for INV); loads w, w^2,
// w^4, w^8 and multiplies the rest (at most three roundings per factor)
template <int R, bool INV>
__device__ __forceinline__ void apply_twiddles(float2* v, const float2* __restrict__ tw, int t1) {
    if constexpr (R == 2) {
        v[1] = cmul(v[1], ldtw<INV>(tw, t1));
    } else if constexpr (R == 4) {
        const float2 w1 = ldtw<INV>(tw, t1), w2 = ldtw<INV>(tw, 2 * t1);
        v[1] = cmul(v[1], w1);
        v[2] = cmul(v[2], w2);
        v[3] = cmul(v[3], cmul(w1, w2));
    } else if constexpr (R == 8) {
        const float2 w1 = ldtw<INV>(tw, t1), w2 = ldtw<INV>(tw, 2 * t1), w4 = ldtw<INV>(tw, 4 * t1);
        const float2 w3 = cmul(w1, w2);
        v[1] = cmul(v[1], w1);
        v[2] = cmul(v[2], w2);
        v[3] = cmul(v[3], w3);
        v[4] = cmul(v[4], w4);
        v[5] = cmul(v[5], cmul(w1, w4));
        v[6] = cmul(v[6], cmul(w2, w4));
        v[7] = cmul(v[7], cmul(w3, w4));
    } else if constexpr (R == 16) {
        const float2 w1 = ldtw<INV>(tw, t1), w2 = ldtw<INV>(tw, 2 * t1);
        const float2 w4 = ldtw<INV>(tw, 4 * t1), w8 = ldtw<INV>(tw, 8 * t1);
        const float2 w3 = cmul(w1, w2), w5 = cmul(w1, w4), w6 = cmul(w2, w4), w7 = cmul(w3, w4);
        v[1] = cmul(v[1], w1);
        v[2] = cmul(v[2], w2);
        v[3] = cmul(v[3], w3);
        v[4] = cmul(v[4], w4);
        v[5] = cmul(v[5], w5);
        v[6] = cmul(v[6], w6);
        v[7] = cmul(v[7], w7);
        v[8] = cmul(v[8], w8);
        v[9] = cmul(v[9], cmul(w1, w8));
        v[10] = cmul(v[10], cmul(w2, w8));
        v[11] = cmul(v[11], cmul(w3, w8));
        v[12] = cmul(v[12], cmul(w4, w8));
        v[13] = cmul(v[13], cmul(w5, w8));
        v[14] = cmul(v[14], cmul(w6, w8));
        v[15] = cmul(v[15], cmul(w7, w8));
    }
}

// ---- odd radices 3, 5, 7 (line lengths R0 * 2^a, the sizes of Sec. 3.3) ----
// cos and sin of 2 pi m / R for R = 3, 5, 7 and m = 0..R-1
__host__ __device__ constexpr float odd_cos(int R, int m) {
    return R == 3 ? (m == 0 ? 1.f : -0.5f)
         : R == 5 ? (m == 0 ? 1.f : (m == 1 || m == 4) ? 0.30901699437494742410f : -0.80901699437494742410f)
         : (m == 0 ? 1.f : (m == 1 || m == 6) ? 0.62348980185873353053f
                          : (m == 2 || m == 5) ? -0.22252093395631440429f : -0.90096886790241912624f);
}
__host__ __device__ constexpr float odd_sin(int R, int m) {
    return R == 3 ? (m == 0 ? 0.f : m == 1 ? 0.86602540378443864676f : -0.86602540378443864676f)
         : R == 5 ? (m == 0 ? 0.f : m == 1 ? 0.95105651629515357212f : m == 2 ? 0.58778525229247312917f
                                  : m == 3 ? -0.58778525229247312917f : -0.95105651629515357212f)
         : (m == 0 ? 0.f : m == 1 ? 0.78183148246802980871f : m == 2 ? 0.97492791218182360702f
                          : m == 3 ? 0.43388373911755812048f : m == 4 ? -0.43388373911755812048f
                          : m == 5 ? -0.97492791218182360702f : -0.78183148246802980871f);
}

// DFT of odd length R in natural order: X[k] = v0 + sum_{r <= H} (v_r + v_{R-r}) cos(2 pi r k/R)
// -/+ i sum_{r <= H} (v_r - v_{R-r}) sin(2 pi r k/R), H = (R-1)/2 (sign - forward, + inverse)
template <int R, bool INV>
__device__ __forceinline__ void dft_odd(float2* v) {
    constexpr int H = (R - 1) / 2;
    float2 sm[H], df[H];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
        sm[r - 1] = cadd(v[r], v[R - r]);
        df[r - 1] = csub(v[r], v[R - r]);
    }
    float2 out[R];
    out[0] = v[0];
#pragma unroll
    for (int r = 0; r < H; ++r) out[0] = cadd(out[0], sm[r]);
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        float2 re = v[0], im = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 1; r <= H; ++r) {
            const int m = (r * k) % R;
            const float c = odd_cos(R, m), sn = odd_sin(R, m);
            re = make_float2(fmaf(c, sm[r - 1].x, re.x), fmaf(c, sm[r - 1].y, re.y));
            im = make_float2(fmaf(sn, df[r - 1].x, im.x), fmaf(sn, df[r - 1].y, im.y));
        }
        // -i*im = (im.y, -im.x), +i*im = (-im.y, im.x)
        const float2 mi = make_float2(im.y, -im.x), pi = make_float2(-im.y, im.x);
        out[k] = cadd(re, INV ? pi : mi);
        out[R - k] = cadd(re, INV ? mi : pi);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = out[k];
}

// In-place FFT of NL lines of length P = R0 * 2^LOGP (R0 = 3, 5 or 7,
// LOGP >= 4) in shared memory at base + l*LS (padded indices): a first Stockham
// pass of radix R0, then radix-16 passes and a trailing radix 2, 4 or 8, with
// twiddles from twm[t] = exp(-2 pi i t / (R0 TWN)).  Threads [0, NL*P/16)
// work (P/16 per line, as for the power-of-two lines); the rest only join the
// barriers.  Called by every thread after the lines are written.  No scaling.
template <int LOGP, int R0, int NL, bool INV>
__device__ __forceinline__ void fft_lines_mixed(float2* base, const float2* __restrict__ twm) {
    constexpr int Q = 1 << LOGP, P = R0 * Q, NB = P / 16, LS = padded_len(P);
    constexpr int TWM = R0 * TWN;
    constexpr int MB = (Q + NB - 1) / NB;          // radix-R0 butterflies per thread (at most)
    const int tid = threadIdx.x;
    const bool active = tid < NL * NB;
    const int line = active ? tid / NB : 0;
    const int j = active ? tid - line * NB : 0;
    float2* a = base + line * LS;
    // pass 0: radix R0, Ns = 1 (no twiddles): inputs b + r Q, outputs b R0 + r
    {
        float2 w[MB][R0];
        if (active) {
#pragma unroll
            for (int q = 0; q < MB; ++q) {
                const int b = j + q * NB;
                if (b < Q) {
#pragma unroll
                    for (int r = 0; r < R0; ++r) w[q][r] = a[pad(b + r * Q)];
                    dft_odd<R0, INV>(w[q]);
                }
            }
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int q = 0; q < MB; ++q) {
                const int b = j + q * NB;
                if (b < Q) {
#pragma unroll
                    for (int r = 0; r < R0; ++r) a[pad(b * R0 + r)] = w[q][r];
                }
            }
        }
        __syncthreads();
    }
    // power-of-two passes with Ns = R0 16^p
    constexpr int N16 = LOGP / 4, REM = 1 << (LOGP % 4);
    float2 v[16];
#pragma unroll
    for (int p = 0; p < N16; ++p) {
        int Ns = R0;
        for (int q = 0; q < p; ++q) Ns *= 16;
        if (active) {
            const int k = j % Ns;
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = a[pad(j + r * NB)];
            apply_twiddles<16, INV>(v, twm, k * (TWM / (Ns * 16)));
            dft<16, INV>(v);
        }
        __syncthreads();
        if (active) {
            const int k = j % Ns;
            const int o = (j - k) * 16 + k;
#pragma unroll
            for (int r = 0; r < 16; ++r) a[pad(o + r * Ns)] = v[r];
        }
        __syncthreads();
    }
    if constexpr (REM > 1) {
        constexpr int RR = REM, NBR = P / RR, PER = 16 / RR;
        int Ns = R0;
        for (int q = 0; q < N16; ++q) Ns *= 16;
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
                const int k = jj % Ns;
                apply_twiddles<RR, INV>(v + b * RR, twm, k * (TWM / (Ns * RR)));
                dft<RR, INV>(v + b * RR);
            }
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int b = 0; b < PER; ++b) {
                const int jj = j + b * NB;
                const int k = jj % Ns;
                const int o = (jj - k) * RR + k;
#pragma unroll
                for (int r = 0; r < RR; ++r) a[pad(o + r * Ns)] = v[b * RR + r];
            }
        }
        __syncthreads();
    }
}

// Main radix of a line of length 2^LOGP and the number of radix-16 passes.// Main radix of a line of length 2^LOGP and the number of radix-16 passes.
template <int LOGP>
struct Plan {
    static constexpr int P = 1 << LOGP;
    static constexpr int R = LOGP >= 4 ? 16 : P;        // registers per thread
    static constexpr int NB = P / R;                    // threads per line
    static constexpr int N16 = LOGP >= 4 ? LOGP / 4 : 0;
    static constexpr int REM = LOGP >= 4 ? (1 << (LOGP % 4)) : 1;   // trailing radix
    static constexpr int LS = padded_len(P);            // line stride in shared memory
};

// In-place FFT of NL lines of length 2^LOGP stored in shared memory at
// base + l*LS (padded indices).  Threads [0, NL*NB) work; the rest only join
// the barriers.  Called by every thread of the block, which must have
// synchronised after writing the lines.  No 1/P scaling.
template <int LOGP, int NL, bool INV>
__device__ __forceinline__ void fft_lines(float2* base, const float2* __restrict__ tw) {
    using PL = Plan<LOGP>;
    constexpr int P = PL::P, R = PL::R, NB = PL::NB, LS = PL::LS;
    const int tid = threadIdx.x;
    const bool active = tid < NL * NB;
    const int line = active ? tid / NB : 0;
    const int j = active ? tid - line * NB : 0;
    float2* a = base + line * LS;
    float2 v[R];

    if constexpr (LOGP == 0) {
        // a length-1 transform is the identity
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
#pragma unroll
        for (int p = 0; p < PL::N16; ++p) {
            const int Ns = 1 << (4 * p);
            if (active) {
                const int k = j & (Ns - 1);
#pragma unroll
                for (int r = 0; r < 16; ++r) v[r] = a[pad(j + r * NB)];
                if (p > 0) apply_twiddles<16, INV>(v, tw, k * (TWN / (Ns * 16)));
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
        }
        if constexpr (PL::REM > 1) {
            constexpr int RR = PL::REM;          // 2, 4 or 8
            constexpr int NBR = P / RR;          // butterflies of radix RR per line
            constexpr int PER = 16 / RR;         // per thread
            constexpr int Ns = 1 << (4 * PL::N16);
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
                    apply_twiddles<RR, INV>(v + b * RR, tw, k * (TWN / (Ns * RR)));
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

// ---------------------------------------------------------------------------
// Radix-8 passes with several lines per thread (used by the column passes).
//
// A thread owns the same butterflies of NC lines (the three field components
// of one column), so a point-wise 3x3 product between components needs no
// shared memory.  Forward transforms use the radix order 8, 8, ..., REM and
// inverse transforms the reversed order REM, 8, ..., 8 (REM = 2^(LOGP mod 3)).
// In Stockham order the last pass of a transform leaves butterfly jj's
// outputs at positions jj + r*P/R - exactly the inputs of a first pass of the
// same radix - so "forward, product, inverse" keeps the data in registers
// across the product.
namespace mmfft {
namespace r8 {

template <int LOGP>
struct Plan8 {
    static constexpr int P = 1 << LOGP;
    static constexpr int N8 = LOGP >= 3 ? LOGP / 3 : 0;
    static constexpr int REM = LOGP >= 3 ? (1 << (LOGP % 3)) : P;
    static constexpr int NPASS = LOGP >= 3 ? N8 + (REM > 1 ? 1 : 0) : (LOGP > 0 ? 1 : 0);
    static constexpr int NB = LOGP >= 3 ? P / 8 : 1;          // threads per line
    static constexpr int LS = padded_len(P);
};

// radix of pass p (REV: reversed order)
template <int LOGP, bool REV>
__host__ __device__ constexpr int radix_at(int p) {
    using PL = Plan8<LOGP>;
    if (LOGP < 3) return PL::P;
    if (PL::REM == 1) return 8;
    if (!REV) return p < PL::N8 ? 8 : PL::REM;
    return p == 0 ? PL::REM : 8;
}
// product of the radices before pass p
template <int LOGP, bool REV>
__host__ __device__ constexpr int ns_at(int p) {
    int ns = 1;
    for (int q = 0; q < p; ++q) ns *= radix_at<LOGP, REV>(q);
    return ns;
}
// butterflies per thread in a pass of radix R
template <int LOGP>
__host__ __device__ constexpr int bpt_of(int R) { return LOGP >= 3 ? 8 / R : 1; }

// position of register value i (= b*R + r) at the input / output of pass PI
template <int LOGP, bool REV, int PI>
__device__ __forceinline__ int in_pos(int j, int i) {
    constexpr int R = radix_at<LOGP, REV>(PI);
    const int b = i / R, r = i - b * R;
    return j + b * Plan8<LOGP>::NB + r * (Plan8<LOGP>::P / R);
}
template <int LOGP, bool REV, int PI>
__device__ __forceinline__ int out_pos(int j, int i) {
    constexpr int R = radix_at<LOGP, REV>(PI), NS = ns_at<LOGP, REV>(PI);
    const int b = i / R, r = i - b * R;
    const int jj = j + b * Plan8<LOGP>::NB, k = jj & (NS - 1);
    return (jj - k) * R + k + r * NS;
}
// number of register values in use
template <int LOGP>
__host__ __device__ constexpr int nval() { return LOGP >= 3 ? 8 : (1 << LOGP); }

// w[r] = tw[t1]^r for r = 1..R-1 (conjugated for INV), formed as in
// apply_twiddles: the loads w, w^2, w^4 and products of them
template <int R, bool INV>
__device__ __forceinline__ void twiddle_powers(float2* w, const float2* __restrict__ tw, int t1) {
    if constexpr (R >= 2) w[1] = ldtw<INV>(tw, t1);
    if constexpr (R >= 4) {
        w[2] = ldtw<INV>(tw, 2 * t1);
        w[3] = cmul(w[1], w[2]);
    }
    if constexpr (R >= 8) {
        w[4] = ldtw<INV>(tw, 4 * t1);
        w[5] = cmul(w[1], w[4]);
        w[6] = cmul(w[2], w[4]);
        w[7] = cmul(w[3], w[4]);
    }
}

// pass PI on the same butterflies of NC lines: the twiddle factors are formed
// once per butterfly and applied to every line
template <int LOGP, bool REV, bool INV, int PI, int NC>
__device__ __forceinline__ void compute_nc(float2 (*v)[8], int j, const float2* __restrict__ tw) {
    constexpr int R = radix_at<LOGP, REV>(PI), NS = ns_at<LOGP, REV>(PI), BPT = bpt_of<LOGP>(R);
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        if constexpr (NS > 1) {
            const int jj = j + b * Plan8<LOGP>::NB, k = jj & (NS - 1);
            float2 w[R > 1 ? R : 2];
            twiddle_powers<R, INV>(w, tw, k * (TWN / (NS * R)));
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int r = 1; r < R; ++r) v[c][b * R + r] = cmul(v[c][b * R + r], w[r]);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) dft<R, INV>(v[c] + b * R);
    }
}
template <int LOGP, bool REV, int PI>
__device__ __forceinline__ void load(const float2* a, float2* v, int j) {
#pragma unroll
    for (int i = 0; i < nval<LOGP>(); ++i) v[i] = a[pad(in_pos<LOGP, REV, PI>(j, i))];
}
template <int LOGP, bool REV, int PI>
__device__ __forceinline__ void store(float2* a, const float2* v, int j) {
#pragma unroll
    for (int i = 0; i < nval<LOGP>(); ++i) a[pad(out_pos<LOGP, REV, PI>(j, i))] = v[i];
}

// Passes PI..NPASS-1 of NC lines held by this thread; on entry the values of
// pass PI's inputs are in shared memory (LOAD = true) or already in registers
// (LOAD = false, only for PI == 0 or straight after the previous pass).  On
// return the last pass's outputs are in registers.  Every thread of the block
// must call it (barriers inside).
template <int LOGP, bool REV, bool INV, int PI, int NC>
__device__ __forceinline__ void run(float2* const* a, float2 (*v)[8], int j, bool active,
                                    const float2* __restrict__ tw, bool from_smem) {
    using PL = Plan8<LOGP>;
    if constexpr (PI < PL::NPASS) {
        if (from_smem) {
            if (active) {
#pragma unroll
                for (int c = 0; c < NC; ++c) load<LOGP, REV, PI>(a[c], v[c], j);
            }
        }
        if (active) compute_nc<LOGP, REV, INV, PI, NC>(v, j, tw);
        if constexpr (PI + 1 < PL::NPASS) {
            __syncthreads();
            if (active) {
#pragma unroll
                for (int c = 0; c < NC; ++c) store<LOGP, REV, PI>(a[c], v[c], j);
            }
            __syncthreads();
            run<LOGP, REV, INV, PI + 1, NC>(a, v, j, active, tw, true);
        }
    }
}

}  // namespace r8
}  // namespace mmfft

// ---------------------------------------------------------------------------
// The register passes of namespace r8 with V values per thread (V = 8 or 16):
// a line of 2^LOGP points takes passes of radix V and one trailing radix
// REM = 2^(LOGP mod log2 V); a pass of radix R < V gives each thread V/R
// butterflies.  Radix 16 halves the shared-memory exchanges of a 2048-point
// line against radix 8 (two instead of three per transform).
namespace mmfft {
namespace rv {

template <int V>
struct Lg { static constexpr int value = V == 16 ? 4 : V == 8 ? 3 : V == 4 ? 2 : 1; };

template <int LOGP, int V>
struct Plan {
    static constexpr int LG = Lg<V>::value;
    static constexpr int P = 1 << LOGP;
    static constexpr int NF = LOGP >= LG ? LOGP / LG : 0;
    static constexpr int REM = LOGP >= LG ? (1 << (LOGP % LG)) : P;
    static constexpr int NPASS = LOGP >= LG ? NF + (REM > 1 ? 1 : 0) : (LOGP > 0 ? 1 : 0);
    static constexpr int NB = LOGP >= LG ? P / V : 1;
    static constexpr int LS = padded_len(P);
    static constexpr int NV = LOGP >= LG ? V : P;
};

template <int LOGP, int V, bool REV>
__host__ __device__ constexpr int radix_at(int p) {
    using PL = Plan<LOGP, V>;
    if (LOGP < PL::LG) return PL::P;
    if (PL::REM == 1) return V;
    if (!REV) return p < PL::NF ? V : PL::REM;
    return p == 0 ? PL::REM : V;
}
template <int LOGP, int V, bool REV>
__host__ __device__ constexpr int ns_at(int p) {
    int ns = 1;
    for (int q = 0; q < p; ++q) ns *= radix_at<LOGP, V, REV>(q);
    return ns;
}
template <int LOGP, int V, bool REV, int PI>
__device__ __forceinline__ int in_pos(int j, int i) {
    constexpr int R = radix_at<LOGP, V, REV>(PI);
    const int b = i / R, r = i - b * R;
    return j + b * Plan<LOGP, V>::NB + r * (Plan<LOGP, V>::P / R);
}
template <int LOGP, int V, bool REV, int PI>
__device__ __forceinline__ int out_pos(int j, int i) {
    constexpr int R = radix_at<LOGP, V, REV>(PI), NS = ns_at<LOGP, V, REV>(PI);
    const int b = i / R, r = i - b * R;
    const int jj = j + b * Plan<LOGP, V>::NB, k = jj & (NS - 1);
    return (jj - k) * R + k + r * NS;
}

// w[r] = tw[t1]^r, r = 1..R-1 (conjugated for INV): loads w, w^2, w^4, w^8, products for the rest
template <int R, bool INV>
__device__ __forceinline__ void twiddle_powers(float2* w, const float2* __restrict__ tw, int t1) {
    if constexpr (R >= 2) w[1] = ldtw<INV>(tw, t1);
    if constexpr (R >= 4) {
        w[2] = ldtw<INV>(tw, 2 * t1);
        w[3] = cmul(w[1], w[2]);
    }
    if constexpr (R >= 8) {
        w[4] = ldtw<INV>(tw, 4 * t1);
        w[5] = cmul(w[1], w[4]);
        w[6] = cmul(w[2], w[4]);
        w[7] = cmul(w[3], w[4]);
    }
    if constexpr (R >= 16) {
        w[8] = ldtw<INV>(tw, 8 * t1);
#pragma unroll
        for (int r = 1; r < 8; ++r) w[8 + r] = cmul(w[r], w[8]);
    }
}

template <int LOGP, int V, bool REV, bool INV, int PI, int NC>
__device__ __forceinline__ void compute_nc(float2 (*v)[V], int j, const float2* __restrict__ tw) {
    constexpr int R = radix_at<LOGP, V, REV>(PI), NS = ns_at<LOGP, V, REV>(PI);
    constexpr int BPT = LOGP >= Plan<LOGP, V>::LG ? V / R : 1;
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        if constexpr (NS > 1) {
            const int jj = j + b * Plan<LOGP, V>::NB, k = jj & (NS - 1);
            float2 w[R > 1 ? R : 2];
            twiddle_powers<R, INV>(w, tw, k * (TWN / (NS * R)));
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int r = 1; r < R; ++r) v[c][b * R + r] = cmul(v[c][b * R + r], w[r]);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) dft<R, INV>(v[c] + b * R);
    }
}
template <int LOGP, int V, bool REV, int PI>
__device__ __forceinline__ void load(const float2* a, float2* v, int j) {
#pragma unroll
    for (int i = 0; i < Plan<LOGP, V>::NV; ++i) v[i] = a[pad(in_pos<LOGP, V, REV, PI>(j, i))];
}
template <int LOGP, int V, bool REV, int PI>
__device__ __forceinline__ void store(float2* a, const float2* v, int j) {
#pragma unroll
    for (int i = 0; i < Plan<LOGP, V>::NV; ++i) a[pad(out_pos<LOGP, V, REV, PI>(j, i))] = v[i];
}

// passes PI..NPASS-1 of NC lines (as r8::run)
template <int LOGP, int V, bool REV, bool INV, int PI, int NC>
__device__ __forceinline__ void run(float2* const* a, float2 (*v)[V], int j, bool active,
                                    const float2* __restrict__ tw, bool from_smem) {
    using PL = Plan<LOGP, V>;
    if constexpr (PI < PL::NPASS) {
        if (from_smem) {
            if (active) {
#pragma unroll
                for (int c = 0; c < NC; ++c) load<LOGP, V, REV, PI>(a[c], v[c], j);
            }
        }
        if (active) compute_nc<LOGP, V, REV, INV, PI, NC>(v, j, tw);
        if constexpr (PI + 1 < PL::NPASS) {
            __syncthreads();
            if (active) {
#pragma unroll
                for (int c = 0; c < NC; ++c) store<LOGP, V, REV, PI>(a[c], v[c], j);
            }
            __syncthreads();
            run<LOGP, V, REV, INV, PI + 1, NC>(a, v, j, active, tw, true);
        }
    }
}

}  // namespace rv
}  // namespace mmfft
