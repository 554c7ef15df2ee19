// hotpath_kernels.cuh - effective field + Landau-Lifshitz step on the GPU (float32):
// the device code, shared by the translation units that instantiate its passes.
//
// One evaluation of H_eff (Sec. 2.1) is the three-stage convolution of
// Sec. 3.2 done as per-axis passes over HBM, each pass a batch of 1-D FFTs in
// shared memory:
//
//   k_xfwd       rows of m (zero padded to Px) -> real-to-complex FFT along x;
//                writes the half spectrum transposed, [c][kx][z][y] (y
//                contiguous), so the next pass reads whole columns.  Padded
//                rows (y >= ny, z >= nz) are never transformed (Sec. 3.2: no
//                FFTs of all-zero arrays).
//   k_colconv    the last transformed axis (y for 2-D grids, z for 3-D
//                grids): forward FFT, point-wise product with the real
//                symmetric kernel (Sec. 3.2), inverse FFT, in one pass; the
//                product happens in registers between the two transforms.
//   k_yfwd, k_yinv   3-D grids only: y forward (writes [c][kx][ky][z]) before
//                and y inverse after the z column pass.
//   k_xinv_local complex-to-real FFT along x, crop, and the whole cell-local
//                remainder of the step fused into its epilogue: exchange
//                (Eq. 3), uniaxial anisotropy (Eq. 4), Zeeman, thermal field
//                (Eq. 6), LL torque (Eq. 1), the Runge-Kutta stage combination
//                (Sec. 2.2), the step-error and torque reductions and, in the
//                last block to finish, the adaptive step controller.
//
// Nothing leaves the device between steps (Sec. 3.1): step size, time, the
// slot holding m_n and the accept decision live in DevState.
#pragma once
#include "mm_internal.cuh"
#include "fft32.cuh"

namespace mm {
using namespace mmfft;
namespace r8 = mmfft::r8;

// Explicit Runge-Kutta tableaus of Sec. 2.2, double precision, by method
// index: 0 Dormand-Prince 5(4) (Dormand & Prince 1980, first same as last),
// 1 Bogacki-Shampine 3(2) (1989, first same as last), 2 Cash-Karp 5(4) (1990),
// 3 classical RK4, 4 Kutta's RK3, 5 Heun-Euler 2(1), 6 Heun (RK2, used when
// the step follows the maximum variation of m).
// c_rka[r][s][j]: weight of k_j in the input of stage s (1-based); with first
// same as last the last stage's row is b.  c_rke[r][j] = b_j - b*_j.
constexpr int NRK = 7;
#define MM_RKA_INIT { \
    {{0}, {0}, {0, 1.0 / 5}, {0, 3.0 / 40, 9.0 / 40}, {0, 44.0 / 45, -56.0 / 15, 32.0 / 9}, \
     {0, 19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729}, \
     {0, 9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656}, \
     {0, 35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}}, \
    {{0}, {0}, {0, 1.0 / 2}, {0, 0.0, 3.0 / 4}, {0, 2.0 / 9, 1.0 / 3, 4.0 / 9}}, \
    {{0}, {0}, {0, 1.0 / 5}, {0, 3.0 / 40, 9.0 / 40}, {0, 3.0 / 10, -9.0 / 10, 6.0 / 5}, \
     {0, -11.0 / 54, 5.0 / 2, -70.0 / 27, 35.0 / 27}, \
     {0, 1631.0 / 55296, 175.0 / 512, 575.0 / 13824, 44275.0 / 110592, 253.0 / 4096}}, \
    {{0}, {0}, {0, 1.0 / 2}, {0, 0.0, 1.0 / 2}, {0, 0.0, 0.0, 1.0}}, \
    {{0}, {0}, {0, 1.0 / 2}, {0, -1.0, 2.0}}, \
    {{0}, {0}, {0, 1.0}}, \
    {{0}, {0}, {0, 1.0}}, \
}
#define MM_RKB_INIT { \
    {0, 35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0.0}, \
    {0, 2.0 / 9, 1.0 / 3, 4.0 / 9, 0.0}, \
    {0, 37.0 / 378, 0.0, 250.0 / 621, 125.0 / 594, 0.0, 512.0 / 1771}, \
    {0, 1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6}, \
    {0, 1.0 / 6, 2.0 / 3, 1.0 / 6}, \
    {0, 1.0 / 2, 1.0 / 2}, \
    {0, 1.0 / 2, 1.0 / 2}, \
}
#define MM_RKE_INIT { \
    {0, 35.0 / 384 - 5179.0 / 57600, 0.0, 500.0 / 1113 - 7571.0 / 16695, 125.0 / 192 - 393.0 / 640, \
     -2187.0 / 6784 + 92097.0 / 339200, 11.0 / 84 - 187.0 / 2100, -1.0 / 40}, \
    {0, 2.0 / 9 - 7.0 / 24, 1.0 / 3 - 1.0 / 4, 4.0 / 9 - 1.0 / 3, -1.0 / 8}, \
    {0, 37.0 / 378 - 2825.0 / 27648, 0.0, 250.0 / 621 - 18575.0 / 48384, 125.0 / 594 - 13525.0 / 55296, \
     -277.0 / 14336, 512.0 / 1771 - 1.0 / 4}, \
    {0}, {0}, \
    {0, 1.0 / 2 - 1.0, 1.0 / 2}, \
    {0}, \
}
static __constant__ double c_rka[NRK][8][8] = MM_RKA_INIT;
static __constant__ double c_rkb[NRK][8] = MM_RKB_INIT;
static __constant__ double c_rke[NRK][8] = MM_RKE_INIT;
// host copies: which stage derivatives a pass must load (stage_need_mask)
static constexpr double h_rka[NRK][8][8] = MM_RKA_INIT;
static constexpr double h_rkb[NRK][8] = MM_RKB_INIT;
static constexpr double h_rke[NRK][8] = MM_RKE_INIT;
// stages, first-same-as-last, exponent denominator q of the step-size factor (0: fixed step)
static __constant__ int c_rks[NRK] = {7, 4, 6, 4, 3, 2, 2};
static __constant__ int c_rkfsal[NRK] = {1, 1, 0, 0, 0, 0, 0};
static __constant__ double c_rkq[NRK] = {5.0, 3.0, 5.0, 0.0, 0.0, 2.0, 0.0};

// ---------------------------------------------------------------------------
// small helpers
struct f3 { float x, y, z; };
__device__ __forceinline__ f3 mk(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 operator*(float s, f3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
// every array a kernel reads through ld3 is read-only for that kernel, so the
// loads may take the non-coherent path and be issued ahead of the stores
__device__ __forceinline__ f3 ld3(const float* __restrict__ a, long long i, long long n) {
    return {__ldg(a + i), __ldg(a + i + n), __ldg(a + i + 2 * n)};
}
__device__ __forceinline__ void st3(float* __restrict__ a, long long i, long long n, f3 v) {
    a[i] = v.x; a[i + n] = v.y; a[i + 2 * n] = v.z;
}
__device__ __forceinline__ f3 normalized(f3 v) {
    float n = sqrtf(dot(v, v));
    float inv = 1.0f / n;
    return inv * v;
}
__device__ __forceinline__ bool finite3(f3 v) { return isfinite(v.x) && isfinite(v.y) && isfinite(v.z); }

// a coefficient c (double) split as hi + lo floats, so that sums like
// m + c k keep the coefficient exact to ~1e-14 (a single-precision c would
// bias every step by the same relative amount)
struct Coef { float hi, lo; };
__device__ __forceinline__ Coef split(double c) {
    float hi = (float)c;
    return {hi, (float)(c - (double)hi)};
}
__device__ __forceinline__ f3 axpy(Coef c, f3 k, f3 acc) {
    return {fmaf(c.lo, k.x, fmaf(c.hi, k.x, acc.x)), fmaf(c.lo, k.y, fmaf(c.hi, k.y, acc.y)),
            fmaf(c.lo, k.z, fmaf(c.hi, k.z, acc.z))};
}

// ---- Philox-4x32-10 (Salmon et al., SC'11) and the Gaussian draw ----------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}
__device__ __forceinline__ float u01(unsigned w) {         // (0,1), exact in float
    return ((float)(w >> 9) + 0.5f) * 1.1920928955078125e-07f;
}
__device__ __forceinline__ f3 gauss3(long long cell, long long step, unsigned long long seed) {
    uint4 w = philox4x32_10(make_uint4((unsigned)cell, (unsigned)step, (unsigned)((unsigned long long)step >> 32), 0u),
                            make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
    float r01 = sqrtf(-2.0f * logf(u01(w.x)));
    float r23 = sqrtf(-2.0f * logf(u01(w.z)));
    float s1, c1, s3, c3;
    sincospif(2.0f * u01(w.y), &s1, &c1);
    sincospif(2.0f * u01(w.w), &s3, &c3);
    return {r01 * c1, r01 * s1, r23 * c3};
}

__device__ __forceinline__ const float* src_ptr(const HotParams& p, int src, int cur) {
    switch (src) {
        case SRC_PTR: return p.m_eval;
        case SRC_CUR: return p.ms[cur];
        case SRC_NEXT: return p.ms[1 - cur];
        case SRC_STAGE1: return p.mstage[1];
        default: return p.mstage[0];      // SRC_STAGE0, SRC_COMBINE2 (materialised)
    }
}

// A block's launch parameters, copied once into shared memory: every field
// the block reads afterwards is a shared-memory load, whether the launch
// covers one sample (ps[0]) or many (ps[sample]).
__device__ __forceinline__ void load_params(const HotParams* __restrict__ src, HotParams* dst) {
    static_assert(sizeof(HotParams) % 4 == 0, "parameter block copied in 32-bit words");
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(HotParams) / 4); i += blockDim.x) d[i] = __ldg(s + i);
    __syncthreads();
}

// FFT lengths for which the x and y passes use the register radix-8 kernels
// (at 4096 points a line needs 512 threads, whose register budget spills:
// the shared-memory radix-16 passes are faster there)
constexpr int XREG_MIN_LOGP = 6, XREG_MAX_LOGP = 11;

// ---------------------------------------------------------------------------
// compile-time shapes of the passes (shared with the host through fft32.cuh)
// x passes: TY rows x 3 components per block; lines of P = R0 * 2^LOGP points
// (R0 = 1, or 3, 5, 7 for the lengths 2^a {3,5,7} of Sec. 3.3), P/16 threads per line
template <int LOGP, int R0 = 1>
struct XS {
    static constexpr int P = R0 << LOGP;
    static constexpr int NBL = R0 == 1 ? nb_of(LOGP) : P / 16;
    static constexpr int TY = 24 * NBL <= 512 ? 16 : 12 * NBL <= 512 ? 8 : 6 * NBL <= 512 ? 4 : 2;
    static constexpr int NL = 3 * TY / 2;       // complex lines (two real rows each)
    static constexpr int NT0 = (NL * NBL + 31) / 32 * 32 < 64 ? 64 : (NL * NBL + 31) / 32 * 32;
    // lines of <= 128 points: 512 threads, more than the transforms use (the
    // rest join their barriers), so that the block's cell epilogue and its
    // loads run about one cell pair per thread instead of several in turn
    // (measured: Dormand-Prince step of the 64 x 16 film 127 -> 107 us).
    // Such grids have few row blocks, so the register budget is not cut for
    // residency.
    static constexpr int NT = (R0 == 1 && LOGP <= 7 && NT0 < 512) ? 512 : NT0;
    static constexpr int LS = padded_len(P);
    static constexpr int HX = P == 1 ? 1 : P / 2 + 1;
    static constexpr int MINB = NT != NT0 || NT >= 768 ? 1 : 1024 / NT;
    static_assert(R0 != 1 || (TY == ty_of(LOGP) && NT0 == threads_of(NL, LOGP)), "power-of-two shapes");
};

// the FFT of the x lines: the power-of-two plan, or a first radix-R0 pass and
// the power-of-two passes (twiddles of the R0 * TWN-entry table twm)
template <int LOGP, int R0, int NL, bool INV>
__device__ __forceinline__ void fft_x_lines(float2* base, const float2* __restrict__ tw, const float2* __restrict__ twm) {
    if constexpr (R0 == 1) fft_lines<LOGP, NL, INV>(base, tw);
    else fft_lines_mixed<LOGP, R0, NL, INV>(base, twm);
}
template <int LOGP, int COLS>
struct CS {                         // column passes: COLS lines x 3 components per block
    static constexpr int P = 1 << LOGP;
    static constexpr int NL = 3 * COLS;
    static constexpr int NT = threads_of(NL, LOGP);
    static constexpr int LS = padded_len(P);
    // 384-thread blocks fit three per SM in 56 registers (measured faster on
    // the 2048-point column pass); other sizes fill ~1024 threads per SM
    static constexpr int MINB = NT >= 768 ? 1 : NT == 384 ? 3 : 1024 / NT;
};

// Half-spectrum unpack of the paired rows of line l (z = a + i b:
// A = (Z_k + conj Z_-k)/2, B = (Z_k - conj Z_-k)/(2i)) and transposed store
// to s1 [c][kx][z][y]: rows 2l, 2l+1 are adjacent y of one component.
template <int LOGP, int R0 = 1>
__device__ __forceinline__ void store_x_spectrum(const HotParams& p, const float2* sm, int y0, int z) {
    using S = XS<LOGP, R0>;
    for (int idx = threadIdx.x; idx < S::NL * S::HX; idx += S::NT) {
        const int l = idx / S::HX, k = idx - l * S::HX;
        const float2 A = sm[l * S::LS + pad(k)];
        const float2 B = cconj(sm[l * S::LS + pad(k == 0 ? 0 : S::P - k)]);
        const float2 D = csub(A, B);
        const float4 out = make_float4(0.5f * (A.x + B.x), 0.5f * (A.y + B.y), 0.5f * D.y, -0.5f * D.x);
        const int c = (2 * l) / S::TY, ty = 2 * l - c * S::TY;
        float2* dst = p.s1 + ((long long)(c * S::HX + k) * p.nz + z) * p.nyp + y0 + ty;
        *reinterpret_cast<float4*>(dst) = out;
    }
}

// x forward pass: rows of m (zero padded to Px) -> R2C -> transposed spectrum.
template <int LOGP, int R0 = 1>
__global__ void __launch_bounds__(XS<LOGP, R0>::NT, XS<LOGP, R0>::MINB) k_xfwd(HotParams p, LaunchArgs a) {
    using S = XS<LOGP, R0>;
    extern __shared__ float2 sm[];
    const int y0 = blockIdx.x * S::TY, z = blockIdx.y;
    DevState* st = p.st;
    if (a.mode != LM_EVAL && st->done) return;
    const int cur = st->cur;
    const long long n = p.ncell;
    const bool comb = a.src == SRC_COMBINE2;
    const float* src = comb ? p.ms[cur] : src_ptr(p, a.src, cur);
    const float* k1 = p.ks[cur];
    float* wout = p.mstage[0];
    const Coef c21 = comb ? split(st->h * c_rka[p.rk][2][1]) : Coef{0.f, 0.f};
    const int NX = p.nx, NY = p.ny;
    // loads of CH items in flight at once, then their combination and stores
    constexpr int NIT = (S::NL * S::P + S::NT - 1) / S::NT;
    constexpr int CH = NIT < 8 ? NIT : 8;
    for (int it0 = 0; it0 < NIT; it0 += CH) {
        float u0[CH], u1[CH], g0[CH], g1[CH];
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            const int idx = threadIdx.x + (it0 + q) * S::NT;
            const int l = idx / S::P, x = idx - l * S::P;
            const int c = (2 * l) / S::TY, ty = 2 * l - c * S::TY;
            const int y = y0 + ty;
            u0[q] = u1[q] = g0[q] = g1[q] = 0.f;
            if (idx < S::NL * S::P && x < NX) {
                const long long i0 = (long long)c * n + ((long long)z * NY + y) * NX + x;
                if (y < NY) { u0[q] = src[i0]; if (comb) g0[q] = k1[i0]; }
                if (y + 1 < NY) { u1[q] = src[i0 + NX]; if (comb) g1[q] = k1[i0 + NX]; }
            }
        }
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            const int idx = threadIdx.x + (it0 + q) * S::NT;
            if (idx >= S::NL * S::P) continue;
            const int l = idx / S::P, x = idx - l * S::P;
            const int c = (2 * l) / S::TY, ty = 2 * l - c * S::TY;
            const int y = y0 + ty;
            float2 v = make_float2(u0[q], u1[q]);
            if (comb && x < NX) {
                const long long i0 = (long long)c * n + ((long long)z * NY + y) * NX + x;
                if (y < NY) { v.x = fmaf(c21.lo, g0[q], fmaf(c21.hi, g0[q], v.x)); wout[i0] = v.x; }
                if (y + 1 < NY) { v.y = fmaf(c21.lo, g1[q], fmaf(c21.hi, g1[q], v.y)); wout[i0 + NX] = v.y; }
            }
            sm[l * S::LS + pad(x)] = v;
        }
    }
    __syncthreads();
    fft_x_lines<LOGP, R0, S::NL, false>(sm, p.tw, p.twr[R0]);
    store_x_spectrum<LOGP, R0>(p, sm, y0, z);
}

// ---------------------------------------------------------------------------
// Column pass with the kernel product in registers (Sec. 3.2 stages i-iii
// along the last transformed axis): forward FFT, product with the real
// symmetric kernel, inverse FFT.  MODE 0: 2-D grids, lines along y of s1
// (kernel components xx yy zz xy; xy odd in ky).  MODE 1: 3-D grids, lines
// along z of s2 (six components; xy, yz odd in ky; xz, yz odd in kz).
// Every thread owns the same radix-8 butterflies of the three components of
// one column; the first forward pass reads global memory directly and the
// last inverse pass writes it directly.
template <int LOGP>
struct CC {
    using PL = r8::Plan8<LOGP>;
    static constexpr int P = PL::P, NB = PL::NB, LS = PL::LS;
    static constexpr int COLS = NB >= 256 ? 1 : (256 / NB > 64 ? 64 : 256 / NB);
    static constexpr int NT = (COLS * NB + 31) / 32 * 32 < 64 ? 64 : (COLS * NB + 31) / 32 * 32;
    static constexpr int LASTF = PL::NPASS > 0 ? PL::NPASS - 1 : 0;
    // resident blocks per SM the compiler is asked for: the default (up to
    // 85 registers for 256 threads) and, for the batched autotuner, a budget
    // of at least 128 registers per thread
    static constexpr int MINB0 = NT <= 256 ? 3 : 1;
    static constexpr int MINB1 = 65536 / (NT * 128) > 0 ? 65536 / (NT * 128) : 1;
};

template <int LOGP, bool REV>
__device__ __forceinline__ int last_out_pos(int j, int i) {
    if constexpr (r8::Plan8<LOGP>::NPASS == 0) return 0;
    else return r8::out_pos<LOGP, REV, CC<LOGP>::LASTF>(j, i);
}

template <int LOGP, int MODE>
__device__ __forceinline__ void colconv_body(const HotParams& p, const LaunchArgs& a, int bx, int by) {
    using S = CC<LOGP>;
    constexpr int NV = r8::nval<LOGP>();
    extern __shared__ float2 sm[];
    if (a.mode != LM_EVAL && p.st->done) return;
    const int tid = threadIdx.x;
    int cl = tid / S::NB;
    const int j = tid - cl * S::NB;
    const bool inblock = cl < S::COLS;
    if (!inblock) cl = 0;
    const int HX = p.hx, PY = p.py;
    int kx, ky = 0, nvalid;
    bool valid;
    long long base, cstride;
    float2* buf;
    if constexpr (MODE == 0) {
        kx = bx * S::COLS + cl;
        valid = kx < HX;
        base = (long long)kx * p.nyp;
        cstride = (long long)HX * p.nyp;
        nvalid = p.ny;
        buf = p.s1;
    } else {
        kx = bx;
        ky = by * S::COLS + cl;
        valid = ky < PY;
        base = ((long long)kx * PY + ky) * p.nzp;
        cstride = (long long)HX * PY * p.nzp;
        nvalid = p.nz;
        buf = p.s2;
    }
    const bool act = inblock && valid;
    float2* lines[3] = {sm + (0 * S::COLS + cl) * S::LS, sm + (1 * S::COLS + cl) * S::LS,
                        sm + (2 * S::COLS + cl) * S::LS};
    float2 v[3][8];
    if (act) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                const int pos = S::PL::NPASS > 0 ? r8::in_pos<LOGP, false, 0>(j, i) : 0;
                v[c][i] = pos < nvalid ? buf[base + c * cstride + pos] : make_float2(0.f, 0.f);
            }
    }
    r8::run<LOGP, false, false, 0, 3>(lines, v, j, act, p.tw, false);
    if (act) {
        const long long cs = (long long)HX * p.hyk * p.hzk;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const int pos = last_out_pos<LOGP, false>(j, i);
            const bool hi = pos > (S::P >> 1);
            const int kq = hi ? S::P - pos : pos;
            const float2 X = v[0][i], Y = v[1][i], Z = v[2][i];
            if constexpr (MODE == 0) {
                const long long b = (long long)kx * p.hyk + kq;
                const float kxx = __ldg(p.kt + b), kyy = __ldg(p.kt + cs + b), kzz = __ldg(p.kt + 2 * cs + b);
                const float kxy = hi ? -__ldg(p.kt + 3 * cs + b) : __ldg(p.kt + 3 * cs + b);
                v[0][i] = make_float2(kxx * X.x + kxy * Y.x, kxx * X.y + kxy * Y.y);
                v[1][i] = make_float2(kxy * X.x + kyy * Y.x, kxy * X.y + kyy * Y.y);
                v[2][i] = make_float2(kzz * Z.x, kzz * Z.y);
            } else {
                const bool yh = ky > (PY >> 1);
                const int kyq = yh ? PY - ky : ky;
                const long long b = ((long long)kx * p.hyk + kyq) * p.hzk + kq;
                const float kxx = __ldg(p.kt + b), kyy = __ldg(p.kt + cs + b), kzz = __ldg(p.kt + 2 * cs + b);
                float kxy = __ldg(p.kt + 3 * cs + b), kxz = __ldg(p.kt + 4 * cs + b), kyz = __ldg(p.kt + 5 * cs + b);
                if (yh) { kxy = -kxy; kyz = -kyz; }
                if (hi) { kxz = -kxz; kyz = -kyz; }
                v[0][i] = make_float2(kxx * X.x + kxy * Y.x + kxz * Z.x, kxx * X.y + kxy * Y.y + kxz * Z.y);
                v[1][i] = make_float2(kxy * X.x + kyy * Y.x + kyz * Z.x, kxy * X.y + kyy * Y.y + kyz * Z.y);
                v[2][i] = make_float2(kxz * X.x + kyz * Y.x + kzz * Z.x, kxz * X.y + kyz * Y.y + kzz * Z.y);
            }
        }
    }
    r8::run<LOGP, true, true, 0, 3>(lines, v, j, act, p.tw, false);
    if (act) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                const int pos = last_out_pos<LOGP, true>(j, i);
                if (pos < nvalid) buf[base + c * cstride + pos] = v[c][i];
            }
    }
}

template <int LOGP, int MODE>
__global__ void __launch_bounds__(CC<LOGP>::NT, CC<LOGP>::NT <= 256 ? 3 : 1) k_colconv(HotParams p, LaunchArgs a) {
    colconv_body<LOGP, MODE>(p, a, blockIdx.x, blockIdx.y);
}
template <int LOGP, int MODE, int V>
__global__ void __launch_bounds__(CC<LOGP>::NT, V ? CC<LOGP>::MINB1 : CC<LOGP>::MINB0)
kb_colconv(const HotParams* __restrict__ ps, const int4* __restrict__ work, LaunchArgs a) {
    const int4 w = work[blockIdx.x];
    __shared__ HotParams s_hp;
    load_params(ps + w.x, &s_hp);
    colconv_body<LOGP, MODE>(s_hp, a, w.y, w.z);
}

// The 2-D column pass with V = 16 register values per thread (radix 16, 16, 8
// for 2048 points: two shared-memory exchanges per transform instead of the
// radix-8 plan's three), one column of three component lines per block.
namespace rv = mmfft::rv;
template <int LOGP>
struct CC16 {
    using PL = rv::Plan<LOGP, 16>;
    static constexpr int P = PL::P, NB = PL::NB, LS = PL::LS, NV = PL::NV;
    static constexpr int NT = NB < 64 ? 64 : NB;
    static constexpr int LASTF = PL::NPASS > 0 ? PL::NPASS - 1 : 0;
};

template <int LOGP>
__global__ void __launch_bounds__(CC16<LOGP>::NT, 3) k_colconv16(HotParams p, LaunchArgs a) {
    using S = CC16<LOGP>;
    constexpr int NV = S::NV;
    extern __shared__ float2 sm[];
    if (a.mode != LM_EVAL && p.st->done) return;
    const int j = threadIdx.x;
    const bool act0 = j < S::NB;
    const int kx = blockIdx.x;
    const int HX = p.hx;
    const bool act = act0 && kx < HX;
    const long long base = (long long)kx * p.nyp, cstride = (long long)HX * p.nyp;
    const int nvalid = p.ny;
    const float2* buf = p.s1;
    float2* lines[3] = {sm, sm + S::LS, sm + 2 * S::LS};
    float2 v[3][16];
    if (act) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                const int pos = rv::in_pos<LOGP, 16, false, 0>(j, i);
                v[c][i] = pos < nvalid ? buf[base + c * cstride + pos] : make_float2(0.f, 0.f);
            }
    }
    rv::run<LOGP, 16, false, false, 0, 3>(lines, v, j, act, p.tw, false);
    if (act) {
        const long long cs = (long long)HX * p.hyk * p.hzk;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const int pos = rv::out_pos<LOGP, 16, false, S::LASTF>(j, i);
            const bool hi = pos > (S::P >> 1);
            const int kq = hi ? S::P - pos : pos;
            const float2 X = v[0][i], Y = v[1][i], Z = v[2][i];
            const long long b = (long long)kx * p.hyk + kq;
            const float kxx = __ldg(p.kt + b), kyy = __ldg(p.kt + cs + b), kzz = __ldg(p.kt + 2 * cs + b);
            const float kxy = hi ? -__ldg(p.kt + 3 * cs + b) : __ldg(p.kt + 3 * cs + b);
            v[0][i] = make_float2(kxx * X.x + kxy * Y.x, kxx * X.y + kxy * Y.y);
            v[1][i] = make_float2(kxy * X.x + kyy * Y.x, kxy * X.y + kyy * Y.y);
            v[2][i] = make_float2(kzz * Z.x, kzz * Z.y);
        }
    }
    rv::run<LOGP, 16, true, true, 0, 3>(lines, v, j, act, p.tw, false);
    if (act) {
        float2* out = p.s1;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                const int pos = rv::out_pos<LOGP, 16, true, S::LASTF>(j, i);
                if (pos < nvalid) out[base + c * cstride + pos] = v[c][i];
            }
    }
}

// ---------------------------------------------------------------------------
// 3-D: y forward pass.  s1 [c][kx][z][y]  ->  s2 [c][kx][ky][z]
// (P < 64: radix-16 shared-memory lines; P >= 64: yfwd_r_body below)
template <int LOGP>
__device__ __forceinline__ void yfwd_body_s(const HotParams& p, const LaunchArgs& a, int bx, int by) {
    constexpr int TZ = tz_of(LOGP);
    using S = CS<LOGP, TZ>;
    extern __shared__ float2 sm[];
    const int kx = bx, z0 = by * TZ;
    if (a.mode != LM_EVAL && p.st->done) return;
    const int HX = p.hx, NY = p.ny, NZ = p.nz;
    for (int idx = threadIdx.x; idx < S::NL * S::P; idx += S::NT) {
        const int l = idx >> LOGP, y = idx & (S::P - 1);
        const int c = l / TZ, zt = l - c * TZ, z = z0 + zt;
        float2 v = make_float2(0.f, 0.f);
        if (y < NY && z < NZ) v = p.s1[((long long)(c * HX + kx) * NZ + z) * p.nyp + y];
        sm[l * S::LS + pad(y)] = v;
    }
    __syncthreads();
    fft_lines<LOGP, S::NL, false>(sm, p.tw);
    for (int idx = threadIdx.x; idx < S::NL * S::P; idx += S::NT) {
        const int zt = idx % TZ, r = idx / TZ, ky = r & (S::P - 1), c = r >> LOGP;
        p.s2[((long long)(c * HX + kx) * S::P + ky) * p.nzp + z0 + zt] = sm[(c * TZ + zt) * S::LS + pad(ky)];
    }
}

// 3-D: y inverse pass.  s2 [c][kx][ky][z]  ->  s1 [c][kx][z][y]
template <int LOGP>
__device__ __forceinline__ void yinv_body_s(const HotParams& p, const LaunchArgs& a, int bx, int by) {
    constexpr int TZ = tz_of(LOGP);
    using S = CS<LOGP, TZ>;
    extern __shared__ float2 sm[];
    const int kx = bx, z0 = by * TZ;
    if (a.mode != LM_EVAL && p.st->done) return;
    const int HX = p.hx, NY = p.ny, NZ = p.nz;
    for (int idx = threadIdx.x; idx < S::NL * S::P; idx += S::NT) {
        const int zt = idx % TZ, r = idx / TZ, ky = r & (S::P - 1), c = r >> LOGP;
        sm[(c * TZ + zt) * S::LS + pad(ky)] = p.s2[((long long)(c * HX + kx) * S::P + ky) * p.nzp + z0 + zt];
    }
    __syncthreads();
    fft_lines<LOGP, S::NL, true>(sm, p.tw);
    for (int idx = threadIdx.x; idx < S::NL * S::P; idx += S::NT) {
        const int l = idx >> LOGP, y = idx & (S::P - 1);
        const int c = l / TZ, zt = l - c * TZ, z = z0 + zt;
        if (y < NY && z < NZ) p.s1[((long long)(c * HX + kx) * NZ + z) * p.nyp + y] = sm[l * S::LS + pad(y)];
    }
}

// 3-D y passes in the register style of the column pass (P >= 64): a block
// holds TZ z lines of one kx; each thread owns the same radix-8 butterflies
// of the three component lines of one z.  The forward pass's first radix-8
// pass reads s1 directly (y contiguous) and its output goes through shared
// memory to the z-contiguous s2; the inverse pass reads s2 through shared
// memory and writes s1 from the registers of its last pass.  TZ equals
// tz_of(LOGP) for these lengths, so the s2 padding and the grid are unchanged.
template <int LOGP>
struct YR {
    using PL = r8::Plan8<LOGP>;
    static constexpr int P = PL::P, NB = PL::NB, LS = PL::LS;
    static constexpr int TZ = NB >= 256 ? 1 : (256 / NB > 8 ? 8 : 256 / NB);
    static constexpr int NT = (TZ * NB + 31) / 32 * 32 < 64 ? 64 : (TZ * NB + 31) / 32 * 32;
    static constexpr int NL = 3 * TZ;
    static constexpr int LASTF = PL::NPASS - 1;
    static constexpr int MINB = NT >= 256 ? 3 : 1024 / NT;
    static constexpr int MINB1 = NT >= 256 ? 3 : 65536 / (NT * 80);   // >= 80 registers (autotuner)
    static constexpr size_t SMEM = (size_t)NL * LS * sizeof(float2);
};

// launch shape of the y passes (either style), shared with the host
template <int LOGP>
struct YS {
    static constexpr bool REG = LOGP >= XREG_MIN_LOGP && LOGP <= XREG_MAX_LOGP;
    static constexpr int TZ = tz_of(LOGP);
    static constexpr int NT = REG ? YR<LOGP>::NT : CS<LOGP, tz_of(LOGP)>::NT;
    static constexpr int MINB = REG ? YR<LOGP>::MINB : CS<LOGP, tz_of(LOGP)>::MINB;
    static constexpr int MINB1 = REG ? YR<LOGP>::MINB1 : CS<LOGP, tz_of(LOGP)>::MINB;
    static constexpr size_t SMEM = REG ? YR<LOGP>::SMEM
                                       : (size_t)CS<LOGP, tz_of(LOGP)>::NL * CS<LOGP, tz_of(LOGP)>::LS * sizeof(float2);
    static_assert(!REG || YR<LOGP>::TZ == tz_of(LOGP), "y tile must match the s2 padding");
};

template <int LOGP>
__device__ __forceinline__ void yfwd_r_body(const HotParams& p, const LaunchArgs& a, int bx, int by) {
    using S = YR<LOGP>;
    extern __shared__ float2 sm[];
    const int kx = bx, z0 = by * S::TZ;
    if (a.mode != LM_EVAL && p.st->done) return;
    const int HX = p.hx, NY = p.ny, NZ = p.nz;
    const int tid = threadIdx.x;
    int zt = tid / S::NB;
    const int j = tid - zt * S::NB;
    const bool act = zt < S::TZ;
    if (!act) zt = 0;
    const int z = z0 + zt;
    float2* lines[3] = {sm + (0 * S::TZ + zt) * S::LS, sm + (1 * S::TZ + zt) * S::LS,
                        sm + (2 * S::TZ + zt) * S::LS};
    float2 v[3][8];
    if (act) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int y = r8::in_pos<LOGP, false, 0>(j, i);
                v[c][i] = (y < NY && z < NZ) ? p.s1[((long long)(c * HX + kx) * NZ + z) * p.nyp + y]
                                             : make_float2(0.f, 0.f);
            }
    }
    r8::run<LOGP, false, false, 0, 3>(lines, v, j, act, p.tw, false);
    __syncthreads();
    if (act) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < 8; ++i) lines[c][pad(r8::out_pos<LOGP, false, S::LASTF>(j, i))] = v[c][i];
    }
    __syncthreads();
    for (int idx = tid; idx < S::NL * S::P; idx += S::NT) {
        const int zz = idx % S::TZ, r = idx / S::TZ, ky = r & (S::P - 1), c = r >> LOGP;
        p.s2[((long long)(c * HX + kx) * S::P + ky) * p.nzp + z0 + zz] = sm[(c * S::TZ + zz) * S::LS + pad(ky)];
    }
}

template <int LOGP>
__device__ __forceinline__ void yinv_r_body(const HotParams& p, const LaunchArgs& a, int bx, int by) {
    using S = YR<LOGP>;
    extern __shared__ float2 sm[];
    const int kx = bx, z0 = by * S::TZ;
    if (a.mode != LM_EVAL && p.st->done) return;
    const int HX = p.hx, NY = p.ny, NZ = p.nz;
    for (int idx = threadIdx.x; idx < S::NL * S::P; idx += S::NT) {
        const int zz = idx % S::TZ, r = idx / S::TZ, ky = r & (S::P - 1), c = r >> LOGP;
        sm[(c * S::TZ + zz) * S::LS + pad(ky)] = p.s2[((long long)(c * HX + kx) * S::P + ky) * p.nzp + z0 + zz];
    }
    __syncthreads();
    const int tid = threadIdx.x;
    int zt = tid / S::NB;
    const int j = tid - zt * S::NB;
    const bool act = zt < S::TZ;
    if (!act) zt = 0;
    const int z = z0 + zt;
    float2* lines[3] = {sm + (0 * S::TZ + zt) * S::LS, sm + (1 * S::TZ + zt) * S::LS,
                        sm + (2 * S::TZ + zt) * S::LS};
    float2 v[3][8];
    r8::run<LOGP, true, true, 0, 3>(lines, v, j, act, p.tw, true);
    if (act && z < NZ) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int y = r8::out_pos<LOGP, true, S::LASTF>(j, i);
                if (y < NY) p.s1[((long long)(c * HX + kx) * NZ + z) * p.nyp + y] = v[c][i];
            }
    }
}

template <int LOGP>
__device__ __forceinline__ void yfwd_body(const HotParams& p, const LaunchArgs& a, int bx, int by) {
    if constexpr (YS<LOGP>::REG) yfwd_r_body<LOGP>(p, a, bx, by);
    else yfwd_body_s<LOGP>(p, a, bx, by);
}
template <int LOGP>
__device__ __forceinline__ void yinv_body(const HotParams& p, const LaunchArgs& a, int bx, int by) {
    if constexpr (YS<LOGP>::REG) yinv_r_body<LOGP>(p, a, bx, by);
    else yinv_body_s<LOGP>(p, a, bx, by);
}


template <int LOGP>
__global__ void __launch_bounds__(YS<LOGP>::NT, YS<LOGP>::MINB)
k_yfwd(HotParams p, LaunchArgs a) {
    yfwd_body<LOGP>(p, a, blockIdx.x, blockIdx.y);
}
template <int LOGP, int V>
__global__ void __launch_bounds__(YS<LOGP>::NT, V ? YS<LOGP>::MINB1 : YS<LOGP>::MINB)
kb_yfwd(const HotParams* __restrict__ ps, const int4* __restrict__ work, LaunchArgs a) {
    const int4 w = work[blockIdx.x];
    __shared__ HotParams s_hp;
    load_params(ps + w.x, &s_hp);
    yfwd_body<LOGP>(s_hp, a, w.y, w.z);
}

template <int LOGP>
__global__ void __launch_bounds__(YS<LOGP>::NT, YS<LOGP>::MINB)
k_yinv(HotParams p, LaunchArgs a) {
    yinv_body<LOGP>(p, a, blockIdx.x, blockIdx.y);
}
template <int LOGP, int V>
__global__ void __launch_bounds__(YS<LOGP>::NT, V ? YS<LOGP>::MINB1 : YS<LOGP>::MINB)
kb_yinv(const HotParams* __restrict__ ps, const int4* __restrict__ work, LaunchArgs a) {
    const int4 w = work[blockIdx.x];
    __shared__ HotParams s_hp;
    load_params(ps + w.x, &s_hp);
    yinv_body<LOGP>(s_hp, a, w.y, w.z);
}

// ---------------------------------------------------------------------------
// Passes along y and z for lengths P = R0 * 2^LOGP with an odd factor R0,
// lines in shared memory (fft_lines_mixed): the column pass (MODE 0: 2-D y
// lines of s1; MODE 1: 3-D z lines of s2) with the kernel product between the
// transforms, and the 3-D y passes.
template <int LOGP, int R0>
struct OS {
    static constexpr int P = R0 << LOGP, NB = P / 16, LS = padded_len(P);
    static constexpr int COLS = cols_of_len(P, 64);
    static constexpr int NL = 3 * COLS;
    static constexpr int NT = (NL * NB + 31) / 32 * 32 < 64 ? 64 : (NL * NB + 31) / 32 * 32;
    static constexpr int TZ = tz_of_len(P);
    static constexpr int NLY = 3 * TZ;
    static constexpr int NTY = (NLY * NB + 31) / 32 * 32 < 64 ? 64 : (NLY * NB + 31) / 32 * 32;
};

template <int LOGP, int R0, int MODE>
__global__ void __launch_bounds__(OS<LOGP, R0>::NT) k_colconv_odd(HotParams p, LaunchArgs a) {
    using S = OS<LOGP, R0>;
    constexpr int P = S::P;
    extern __shared__ float2 sm[];
    if (a.mode != LM_EVAL && p.st->done) return;
    const int HX = p.hx, PY = p.py;
    const long long cstride = MODE == 0 ? (long long)HX * p.nyp : (long long)HX * PY * p.nzp;
    const int nvalid = MODE == 0 ? p.ny : p.nz;
    float2* buf = MODE == 0 ? p.s1 : p.s2;
    // line base of column cl of this block (valid or not)
    auto col = [&](int cl, long long& base) {
        if (MODE == 0) {
            const int kx = blockIdx.x * S::COLS + cl;
            base = (long long)kx * p.nyp;
            return kx < HX;
        }
        const int ky = blockIdx.y * S::COLS + cl;
        base = ((long long)blockIdx.x * PY + ky) * p.nzp;
        return ky < PY;
    };
    for (int idx = threadIdx.x; idx < S::NL * P; idx += S::NT) {
        const int l = idx / P, pos = idx - l * P;
        const int c = l / S::COLS, cl = l - c * S::COLS;
        long long base;
        const bool ok = col(cl, base);
        sm[l * S::LS + pad(pos)] = (ok && pos < nvalid) ? buf[base + c * cstride + pos] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_lines_mixed<LOGP, R0, S::NL, false>(sm, p.twr[R0]);
    {
        const long long cs = (long long)HX * p.hyk * p.hzk;
        for (int idx = threadIdx.x; idx < S::COLS * P; idx += S::NT) {
            const int cl = idx / P, k = idx - cl * P;
            long long base;
            if (!col(cl, base)) continue;
            const bool hi = k > (P >> 1);
            const int kq = hi ? P - k : k;
            float2* e0 = sm + (0 * S::COLS + cl) * S::LS + pad(k);
            float2* e1 = sm + (1 * S::COLS + cl) * S::LS + pad(k);
            float2* e2 = sm + (2 * S::COLS + cl) * S::LS + pad(k);
            const float2 X = *e0, Y = *e1, Z = *e2;
            if constexpr (MODE == 0) {
                const long long b = (long long)(blockIdx.x * S::COLS + cl) * p.hyk + kq;
                const float kxx = __ldg(p.kt + b), kyy = __ldg(p.kt + cs + b), kzz = __ldg(p.kt + 2 * cs + b);
                const float kxy = hi ? -__ldg(p.kt + 3 * cs + b) : __ldg(p.kt + 3 * cs + b);
                *e0 = make_float2(kxx * X.x + kxy * Y.x, kxx * X.y + kxy * Y.y);
                *e1 = make_float2(kxy * X.x + kyy * Y.x, kxy * X.y + kyy * Y.y);
                *e2 = make_float2(kzz * Z.x, kzz * Z.y);
            } else {
                const int kx = blockIdx.x, ky = blockIdx.y * S::COLS + cl;
                const bool yh = ky > (PY >> 1);
                const int kyq = yh ? PY - ky : ky;
                const long long b = ((long long)kx * p.hyk + kyq) * p.hzk + kq;
                const float kxx = __ldg(p.kt + b), kyy = __ldg(p.kt + cs + b), kzz = __ldg(p.kt + 2 * cs + b);
                float kxy = __ldg(p.kt + 3 * cs + b), kxz = __ldg(p.kt + 4 * cs + b), kyz = __ldg(p.kt + 5 * cs + b);
                if (yh) { kxy = -kxy; kyz = -kyz; }
                if (hi) { kxz = -kxz; kyz = -kyz; }
                *e0 = make_float2(kxx * X.x + kxy * Y.x + kxz * Z.x, kxx * X.y + kxy * Y.y + kxz * Z.y);
                *e1 = make_float2(kxy * X.x + kyy * Y.x + kyz * Z.x, kxy * X.y + kyy * Y.y + kyz * Z.y);
                *e2 = make_float2(kxz * X.x + kyz * Y.x + kzz * Z.x, kxz * X.y + kyz * Y.y + kzz * Z.y);
            }
        }
    }
    __syncthreads();
    fft_lines_mixed<LOGP, R0, S::NL, true>(sm, p.twr[R0]);
    for (int idx = threadIdx.x; idx < S::NL * P; idx += S::NT) {
        const int l = idx / P, pos = idx - l * P;
        const int c = l / S::COLS, cl = l - c * S::COLS;
        long long base;
        if (col(cl, base) && pos < nvalid) buf[base + c * cstride + pos] = sm[l * S::LS + pad(pos)];
    }
}

// 3-D y forward (s1 [c][kx][z][y] -> s2 [c][kx][ky][z]) and inverse passes, TZ z lines of one kx
template <int LOGP, int R0, bool INV>
__global__ void __launch_bounds__(OS<LOGP, R0>::NTY) k_ypass_odd(HotParams p, LaunchArgs a) {
    using S = OS<LOGP, R0>;
    constexpr int P = S::P, TZ = S::TZ;
    extern __shared__ float2 sm[];
    const int kx = blockIdx.x, z0 = blockIdx.y * TZ;
    if (a.mode != LM_EVAL && p.st->done) return;
    const int HX = p.hx, NY = p.ny, NZ = p.nz;
    if (!INV) {
        for (int idx = threadIdx.x; idx < S::NLY * P; idx += S::NTY) {
            const int l = idx / P, y = idx - l * P;
            const int c = l / TZ, zt = l - c * TZ, z = z0 + zt;
            float2 v = make_float2(0.f, 0.f);
            if (y < NY && z < NZ) v = p.s1[((long long)(c * HX + kx) * NZ + z) * p.nyp + y];
            sm[l * S::LS + pad(y)] = v;
        }
    } else {
        for (int idx = threadIdx.x; idx < S::NLY * P; idx += S::NTY) {
            const int zt = idx % TZ, r = idx / TZ, ky = r % P, c = r / P;
            sm[(c * TZ + zt) * S::LS + pad(ky)] = p.s2[((long long)(c * HX + kx) * P + ky) * p.nzp + z0 + zt];
        }
    }
    __syncthreads();
    fft_lines_mixed<LOGP, R0, S::NLY, INV>(sm, p.twr[R0]);
    if (!INV) {
        for (int idx = threadIdx.x; idx < S::NLY * P; idx += S::NTY) {
            const int zt = idx % TZ, r = idx / TZ, ky = r % P, c = r / P;
            p.s2[((long long)(c * HX + kx) * P + ky) * p.nzp + z0 + zt] = sm[(c * TZ + zt) * S::LS + pad(ky)];
        }
    } else {
        for (int idx = threadIdx.x; idx < S::NLY * P; idx += S::NTY) {
            const int l = idx / P, y = idx - l * P;
            const int c = l / TZ, zt = l - c * TZ, z = z0 + zt;
            if (y < NY && z < NZ) p.s1[((long long)(c * HX + kx) * NZ + z) * p.nyp + y] = sm[l * S::LS + pad(y)];
        }
    }
}

// ---------------------------------------------------------------------------
// block reduction + last-block step control
struct Partials {
    float err, torque;
    double energy;
    double tsq;           // sum |m x h|^2 (EVAL mode with energy): the damping dissipation
    unsigned bad;
};

static __device__ void finalize(const HotParams& p, const LaunchArgs& a) {
    DevState* st = p.st;
    const float err = __uint_as_float(atomicExch(&st->err_bits, 0u));
    const float tq = __uint_as_float(atomicExch(&st->torque_bits, 0u));
    const unsigned bad = atomicExch(&st->bad, 0u);
    st->blocks_done = 0u;
    // the stage passes before the last one have no last block (reduce_and_finish):
    // the last pass counts their evaluations too
    st->evals += (a.mode == LM_RKFINAL) ? p.rk_stages - 1 : (a.mode == LM_HEUN2) ? 2 : 1;
    switch (a.mode) {
        case LM_EVAL:
            st->max_torque = tq;
            if (bad) st->status = -5;
            break;
        case LM_K1:
            st->max_torque = tq;
            if (bad) { st->status = -5; st->done = 1; }
            else if (st->torque_tol > 0.0 && tq < st->torque_tol) st->done = 1;
            if (st->max_dm > 0.0 && !st->done) {
                // fixed maximum variation of m per step: the fastest cell moves
                // by max_dm to first order (err = max |k1|)
                double hn = err > 0.0f ? st->max_dm / (double)err : st->h_cap;
                if (st->h_cap > 0.0 && !(hn <= st->h_cap)) hn = st->h_cap;
                if (hn > 0.0) st->h = hn;
            }
            break;
        case LM_RKFINAL: {
            st->last_err = err;
            // a tableau whose last stage is not the new state evaluates the
            // field at a stage point: its torque says nothing about m_{n+1}.
            // The next step's k1 pass (at the accepted state) takes the
            // torque decision instead.
            const bool tq_here = p.rk_fsal != 0;
            if (bad || !isfinite(err)) { st->status = -5; st->done = 1; break; }
            const double q = c_rkq[p.rk];
            const bool fixed = st->fixed_h || q == 0.0;
            const bool accept = fixed || (double)err <= st->tol;
            double f = (err == 0.0f) ? 5.0 : 0.9 * pow(st->tol / (double)err, 1.0 / (q > 0.0 ? q : 5.0));
            f = fmin(fmax(f, 0.2), 5.0);
            if (fixed) f = 1.0;
            if (accept) {
                if (st->after_reject) f = fmin(f, 1.0);
                st->t += st->h;
                st->cur ^= 1;
                st->accepted += 1;
                st->step_index += 1;
                if (tq_here) st->max_torque = tq;
                st->after_reject = 0;
            } else {
                f = fmin(f, 1.0);
                st->rejected += 1;
                st->after_reject = 1;
            }
            st->h *= f;
            if (st->t_end > 0.0) {
                const double left = st->t_end - st->t;
                if (left <= 1e-12 * st->t_end) st->done = 1;
                else st->h = fmin(st->h, left);
            }
            if (tq_here && accept && st->torque_tol > 0.0 && tq < st->torque_tol) st->done = 1;
            if (!st->done && st->h < st->h_min) { st->status = -4; st->done = 1; }
            break;
        }
        case LM_EULER:
        case LM_HEUN2:
            if (bad) { st->status = -5; st->done = 1; break; }
            // tq = max |m x h| at m_n (the Euler pass, or Heun's first stage).
            // Below the bound the run stops at m_n: the new state just written
            // to the other slot is not taken, and time does not advance.
            st->max_torque = tq;
            if (st->torque_tol > 0.0 && tq < st->torque_tol) { st->done = 1; break; }
            st->t += p.dt_d;
            st->cur ^= 1;
            st->step_index += 1;
            st->accepted += 1;
            if (st->t_end > 0.0 && st->t >= st->t_end * (1.0 - 1e-12)) st->done = 1;
            break;
        default:
            if (bad) { st->status = -5; st->done = 1; }
            break;
    }
}

// nblk: the blocks of this evaluation that report (the last of them runs finalize).
// EV = false: a pass that never runs in evaluation mode (no energy sums).
template <bool EV = true>
__device__ void reduce_and_finish(const HotParams& p, const LaunchArgs& a, Partials pt, int nblk) {
    if (a.mode == LM_RK) {
        // intermediate stages reduce nothing but the non-finite flag, which the
        // step's last pass reads: one vote per warp, an atomic only when set
        if (__any_sync(0xffffffffu, pt.bad) && (threadIdx.x & 31) == 0) atomicOr(&p.st->bad, 1u);
        return;
    }
    // Heun's first stage evaluates m_n: it reduces the torque there (one atomic
    // per block) for the second stage's last block, which stops the run on it
    const bool last_pass = a.mode != LM_HEUN1;
    __shared__ float r_err[32], r_tq[32];
    __shared__ double r_e[32], r_t[32];
    __shared__ unsigned r_bad[32];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pt.err = fmaxf(pt.err, __shfl_xor_sync(0xffffffffu, pt.err, o));
        pt.torque = fmaxf(pt.torque, __shfl_xor_sync(0xffffffffu, pt.torque, o));
        if constexpr (EV) {
            pt.energy += __shfl_xor_sync(0xffffffffu, pt.energy, o);
            pt.tsq += __shfl_xor_sync(0xffffffffu, pt.tsq, o);
        }
        pt.bad |= __shfl_xor_sync(0xffffffffu, pt.bad, o);
    }
    if (lane == 0) { r_err[wid] = pt.err; r_tq[wid] = pt.torque; r_e[wid] = pt.energy; r_t[wid] = pt.tsq; r_bad[wid] = pt.bad; }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 1; w < nw; ++w) {
            pt.err = fmaxf(pt.err, r_err[w]);
            pt.torque = fmaxf(pt.torque, r_tq[w]);
            if constexpr (EV) {
                pt.energy += r_e[w];
                pt.tsq += r_t[w];
            }
            pt.bad |= r_bad[w];
        }
        DevState* st = p.st;
        if (pt.err > 0.f) atomicMax(&st->err_bits, __float_as_uint(pt.err));
        if (pt.torque > 0.f) atomicMax(&st->torque_bits, __float_as_uint(pt.torque));
        if (EV && a.mode == LM_EVAL && p.want_energy) {
            atomicAdd(&st->energy_acc, pt.energy);
            atomicAdd(&st->tsq_acc, pt.tsq);
        }
        if (pt.bad) atomicOr(&st->bad, 1u);
        s_last = 0;
        if (last_pass) {
            __threadfence();
            const unsigned prev = atomicAdd(&st->blocks_done, 1u);
            s_last = (prev == (unsigned)nblk - 1u);
        }
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        finalize(p, a);
    }
}

// ---------------------------------------------------------------------------
// Everything that happens to one cell once its demag field is known.
struct StageCoefs {
    Coef c[8];          // per mode: stage combination weights (see stage_coefs)
    Coef e[8];          // final stage: error weights h (b_j - b*_j)
};

// What one cell reads: m at the cell and its neighbours (a missing neighbour
// is the cell itself) and the stage inputs q0 = m_n, qk[j-1] = k_j.
struct CellIn {
    f3 m, mxp, mxm, myp, mym, mzp, mzm;
    f3 q0;
    f3 qk[6];
    f3 u;             // easy axis of this cell
};

// Issues every load a cell needs, before any arithmetic, so their latencies
// overlap.  Which k_j are read is fixed by the tableau (a.need), not by h.
// LITE: the film's common term set (no z neighbours, one easy axis, no cubic
// anisotropy, no thermal field, no spin-transfer torque) compiled without the
// other terms' registers; the host selects it only when that holds.
template <bool LITE = false>
__device__ __forceinline__ void load_cell(const HotParams& p, const LaunchArgs& a, int cur,
                                          const float* __restrict__ min, long long cell, int x, int y, int z,
                                          CellIn& in) {
    const long long n = p.ncell;
    // neighbour indices; a missing neighbour (free boundary) points at the cell
    // itself, so its difference is zero
    long long ixp = cell, ixm = cell;
    if (x + 1 < p.nx) ixp = cell + 1;
    else if (p.pbc[0]) ixp = cell - (p.nx - 1);
    if (x > 0) ixm = cell - 1;
    else if (p.pbc[0]) ixm = cell + (p.nx - 1);
    const bool usey = p.ny > 1 || p.pbc[1];
    const bool usez = !LITE && (p.nz > 1 || p.pbc[2]);
    long long iyp = cell, iym = cell, izp = cell, izm = cell;
    if (usey) {
        const long long sy = p.nx;
        if (y + 1 < p.ny) iyp = cell + sy;
        else if (p.pbc[1]) iyp = cell - (long long)(p.ny - 1) * sy;
        if (y > 0) iym = cell - sy;
        else if (p.pbc[1]) iym = cell + (long long)(p.ny - 1) * sy;
    }
    if (usez) {
        const long long sz = (long long)p.nx * p.ny;
        if (z + 1 < p.nz) izp = cell + sz;
        else if (p.pbc[2]) izp = cell - (long long)(p.nz - 1) * sz;
        if (z > 0) izm = cell - sz;
        else if (p.pbc[2]) izm = cell + (long long)(p.nz - 1) * sz;
    }
    in.m = ld3(min, cell, n);
    in.mxp = ld3(min, ixp, n);
    in.mxm = ld3(min, ixm, n);
    in.myp = in.mym = in.mzp = in.mzm = in.m;
    if (usey) { in.myp = ld3(min, iyp, n); in.mym = ld3(min, iym, n); }
    if (usez) { in.mzp = ld3(min, izp, n); in.mzm = ld3(min, izm, n); }
    in.u = (!LITE && p.uaxis) ? ld3(p.uaxis, cell, n) : mk(p.ux, p.uy, p.uz);
    in.q0 = mk(0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 6; ++j) in.qk[j] = in.q0;
    const int s = a.stage;
    switch (a.mode) {
        case LM_RK:                                  // stage s: input of s+1 = m_n + sum_{j<=s} a k_j
            in.q0 = ld3(p.ms[cur], cell, n);
            in.qk[0] = ld3(p.ks[cur], cell, n);
#pragma unroll
            for (int j = 2; j <= 6; ++j)
                if (j < s && ((a.need >> j) & 1)) in.qk[j - 1] = ld3(p.kb[j], cell, n);
            break;
        case LM_RKFINAL:                             // stage S: error (and m_{n+1} without FSAL)
            if (!p.rk_fsal) in.q0 = ld3(p.ms[cur], cell, n);
            in.qk[0] = ld3(p.ks[cur], cell, n);
#pragma unroll
            for (int j = 2; j <= 6; ++j)
                if (j < s && ((a.need >> j) & 1)) in.qk[j - 1] = ld3(p.kb[j], cell, n);
            break;
        case LM_HEUN2:
            in.q0 = ld3(p.ms[cur], cell, n);
            in.qk[0] = ld3(p.ks[cur], cell, n);
            break;
        default: break;
    }
}

// Everything that happens to one cell once its inputs and demag field are
// known.  Returns the magnetisation the next evaluation of this step reads at
// this cell (m_{s+1}, m_2, the predictor or m_{n+1}); zero when there is none.
template <bool EV = true, bool LITE = false>
__device__ __forceinline__ f3 update_cell(const HotParams& p, const LaunchArgs& a, int cur, const StageCoefs& sc,
                                          long long cell, const CellIn& in, f3 hd, long long tstep, Partials& pt) {
    const long long n = p.ncell;
    const f3 m = in.m, mxp = in.mxp, mxm = in.mxm, myp = in.myp, mym = in.mym, mzp = in.mzp, mzm = in.mzm;
    const f3 q0 = in.q0;
    const f3* qk = in.qk;
    const bool usey = p.ny > 1 || p.pbc[1];
    const bool usez = !LITE && (p.nz > 1 || p.pbc[2]);
    const int s = a.stage;
    const bool fsal = p.rk_fsal != 0;
    // exchange, 6-neighbour (4 in 2-D) Laplacian (Eq. 3)
    f3 hex = p.cex[0] * ((mxp - m) + (mxm - m));
    if (usey) hex = hex + p.cex[1] * ((myp - m) + (mym - m));
    if (usez) hex = hex + p.cex[2] * ((mzp - m) + (mzm - m));
    const f3 u = in.u;
    f3 han = (p.kan * dot(m, u)) * u;
    float ecub = 0.f;
    if (!LITE && (p.kc1 != 0.f || p.kc2 != 0.f)) {
        // cubic anisotropy (Eq. 5): h = -sum_i a_i [kc1 (a_j^2 + a_k^2) + kc2 a_j^2 a_k^2] c_i
        const f3 c1 = mk(p.c[0][0], p.c[0][1], p.c[0][2]);
        const f3 c2 = mk(p.c[1][0], p.c[1][1], p.c[1][2]);
        const f3 c3 = mk(p.c[2][0], p.c[2][1], p.c[2][2]);
        const float a1 = dot(m, c1), a2 = dot(m, c2), a3 = dot(m, c3);
        const float s1 = a1 * a1, s2 = a2 * a2, s3 = a3 * a3;
        han = han - ((a1 * (p.kc1 * (s2 + s3) + p.kc2 * s2 * s3)) * c1 +
                     (a2 * (p.kc1 * (s1 + s3) + p.kc2 * s1 * s3)) * c2 +
                     (a3 * (p.kc1 * (s1 + s2) + p.kc2 * s1 * s2)) * c3);
        ecub = 0.5f * (p.kc1 * (s1 * s2 + s2 * s3 + s1 * s3) + p.kc2 * s1 * s2 * s3);   // phi/(mu0 Ms^2)
    }
    const f3 hz = mk(p.hzx, p.hzy, p.hzz);
    f3 h = hd + hex + han + hz;
    if (!LITE && p.sigma_th > 0.f) h = h + p.sigma_th * gauss3(cell, tstep, p.seed);
    const f3 mxh = cross(m, h);
    f3 k = (-p.llpref) * (mxh + p.alpha * cross(m, mxh));
    if (!LITE && p.stt) {
        // Zhang-Li spin-transfer torque (Eq. 7 / Ms): (j.grad)m from the same
        // neighbours (a missing one is the cell itself), b_j folded into stt_s
        const f3 us = (p.stt_s[0] * (mxp - mxm) + p.stt_s[1] * (myp - mym)) + p.stt_s[2] * (mzp - mzm);
        const f3 mxu = cross(m, us);
        k = k - p.llpref * (cross(m, mxu) + p.stt_beta * mxu);
    }
    const float tq = sqrtf(dot(mxh, mxh));
    f3 next = mk(0.f, 0.f, 0.f);

    switch (a.mode) {
        case LM_EVAL: {
            if constexpr (!EV) break;
            if (p.h_out) st3(p.h_out, cell, n, p.h_scale * h);
            if (p.tq_out) st3(p.tq_out, cell, n, p.t_scale * k);
            pt.torque = fmaxf(pt.torque, tq);
            if (p.want_energy) {
                // quadratic terms as -m.H/2; the quartic cubic term by its density
                const f3 hquad = hd + hex + (p.kan * dot(m, u)) * u;
                pt.energy += -0.5 * (double)dot(m, hquad) - (double)dot(m, hz) + (double)ecub;
                pt.tsq += (double)dot(mxh, mxh);
            }
            pt.bad |= !finite3(h);
            break;
        }
        case LM_K1:
            st3(p.ks[cur], cell, n, k);
            pt.torque = fmaxf(pt.torque, tq);
            pt.err = fmaxf(pt.err, sqrtf(dot(k, k)));    // max |dm/dt| (maximum-variation steps)
            pt.bad |= !finite3(k);
            next = axpy(sc.c[1], k, m);                 // m_2 = m_n + h a21 k1
            st3(p.mstage[0], cell, n, next);
            break;
        case LM_RK: {                                    // stages 2..S-1
            st3(p.kb[s], cell, n, k);
            f3 acc = axpy(sc.c[1], qk[0], q0);
#pragma unroll
            for (int j = 2; j <= 6; ++j)
                if (j < s && sc.c[j].hi != 0.f) acc = axpy(sc.c[j], qk[j - 1], acc);
            acc = axpy(sc.c[s], k, acc);
            if (fsal && s + 1 == p.rk_stages) {          // the last stage evaluates the candidate
                next = normalized(acc);
                st3(p.ms[1 - cur], cell, n, next);
            } else {
                st3(p.mstage[(s + 1) & 1], cell, n, acc);
                next = acc;
            }
            pt.bad |= !finite3(k);
            break;
        }
        case LM_RKFINAL: {                               // stage S
            f3 e = mk(0.f, 0.f, 0.f);
            e = axpy(sc.e[1], qk[0], e);
#pragma unroll
            for (int j = 2; j <= 6; ++j)
                if (j < s && sc.e[j].hi != 0.f) e = axpy(sc.e[j], qk[j - 1], e);
            e = axpy(sc.e[s], k, e);
            if (fsal) {
                st3(p.ks[1 - cur], cell, n, k);          // k_S = f(m_{n+1}) is the next step's k1
            } else {
                f3 acc = axpy(sc.c[1], qk[0], q0);
#pragma unroll
                for (int j = 2; j <= 6; ++j)
                    if (j < s && sc.c[j].hi != 0.f) acc = axpy(sc.c[j], qk[j - 1], acc);
                acc = axpy(sc.c[s], k, acc);
                const f3 mn = normalized(acc);
                st3(p.ms[1 - cur], cell, n, mn);
                pt.bad |= !finite3(mn);
            }
            pt.err = fmaxf(pt.err, sqrtf(dot(e, e)));
            pt.torque = fmaxf(pt.torque, tq);
            pt.bad |= !finite3(k) || !finite3(e);
            break;
        }
        case LM_EULER: {
            next = normalized(axpy(sc.c[0], k, m));
            st3(p.ms[1 - cur], cell, n, next);
            pt.torque = fmaxf(pt.torque, tq);           // at m_n
            pt.bad |= !finite3(next);
            break;
        }
        case LM_HEUN1: {
            st3(p.ks[cur], cell, n, k);
            next = axpy(sc.c[0], k, m);
            st3(p.mstage[0], cell, n, next);
            pt.torque = fmaxf(pt.torque, tq);           // at m_n
            pt.bad |= !finite3(k);
            break;
        }
        case LM_HEUN2: {
            f3 acc = axpy(sc.c[0], qk[0], q0);
            acc = axpy(sc.c[0], k, acc);
            next = normalized(acc);
            st3(p.ms[1 - cur], cell, n, next);
            pt.bad |= !finite3(next);
            break;
        }
        default: break;
    }
    return next;
}

template <bool LITE = false>
__device__ __forceinline__ f3 cell_update(const HotParams& p, const LaunchArgs& a, int cur, const StageCoefs& sc,
                                          const float* __restrict__ min, long long cell, int x, int y, int z,
                                          f3 hd, long long tstep, Partials& pt) {
    CellIn in;
    load_cell<LITE>(p, a, cur, min, cell, x, y, z, in);
    return update_cell<true, LITE>(p, a, cur, sc, cell, in, hd, tstep, pt);
}

// The stage weights of this pass times h, split into float pairs.  Called by
// the first warp of a block: lane l < 8 forms c[l], lane 8 + l forms e[l].
static __device__ void stage_coefs(const HotParams& p, const LaunchArgs& a, const DevState* st, StageCoefs& sc) {
    const int lane = threadIdx.x & 31;
    if (lane >= 16) return;
    const int j = lane & 7;
    const bool err = lane >= 8;
    const double h = st->h;
    const int r = p.rk;
    double v = 0.0;
    switch (a.mode) {
        case LM_K1:
            if (!err && j == 1) v = h * c_rka[r][2][1];
            break;
        case LM_RK:
            if (!err && j >= 1 && j <= a.stage) v = h * c_rka[r][a.stage + 1][j];
            break;
        case LM_RKFINAL:
            if (j >= 1) v = h * (err ? c_rke[r][j] : c_rkb[r][j]);
            break;
        case LM_EULER:
        case LM_HEUN1:
            if (!err && j == 0) v = p.dt_d;
            break;
        case LM_HEUN2:
            if (!err && j == 0) v = 0.5 * p.dt_d;
            break;
        default: break;
    }
    const Coef c = v == 0.0 ? Coef{0.f, 0.f} : split(v);
    if (err) sc.e[j] = c;
    else sc.c[j] = c;
}


// Inverse x pass (C2R) + crop + cell-local epilogue.  With FUSE the block
// then transforms the next evaluation's input for its rows (forward R2C,
// transposed store), so the next stage needs no separate x-forward pass.
// The spectrum region a block reads is exactly the region it writes.
template <int LOGP, bool FUSE, bool LITE = false, int R0 = 1>
__global__ void __launch_bounds__(XS<LOGP, R0>::NT, XS<LOGP, R0>::MINB) k_xinv_local(HotParams p, LaunchArgs a) {
    using S = XS<LOGP, R0>;
    constexpr int HP = S::TY / 2;                 // row pairs per block
    extern __shared__ float2 sm[];
    __shared__ StageCoefs s_sc;
    __shared__ int s_cur;
    __shared__ long long s_tstep;
    const int y0 = blockIdx.x * S::TY, z = blockIdx.y;
    DevState* st = p.st;
    if (a.mode != LM_EVAL && st->done) return;
    if (threadIdx.x < 32) stage_coefs(p, a, st, s_sc);
    if (threadIdx.x == 0) {
        s_cur = st->cur;
        s_tstep = (a.mode == LM_EVAL) ? p.thermal_step : st->step_index;
    }
    {
        // every load of the block's spectrum in flight at once, then the unpack
        constexpr int NLD = (S::NL * S::HX + S::NT - 1) / S::NT;
        float4 vv[NLD];
#pragma unroll
        for (int it = 0; it < NLD; ++it) {
            const int idx = threadIdx.x + it * S::NT;
            if (idx < S::NL * S::HX) {
                const int l = idx / S::HX, k = idx - l * S::HX;
                const int c = (2 * l) / S::TY, ty = 2 * l - c * S::TY;
                vv[it] = *reinterpret_cast<const float4*>(
                    p.s1 + ((long long)(c * S::HX + k) * p.nz + z) * p.nyp + y0 + ty);
            }
        }
#pragma unroll
        for (int it = 0; it < NLD; ++it) {
            const int idx = threadIdx.x + it * S::NT;
            if (idx < S::NL * S::HX) {
                const int l = idx / S::HX, k = idx - l * S::HX;
                const float4 v = vv[it];
                // Z = A + iB with A = (v.x, v.y), B = (v.z, v.w); Z[-k] = conj(A) + i conj(B)
                sm[l * S::LS + pad(k)] = make_float2(v.x - v.w, v.y + v.z);
                if (k > 0 && 2 * k < S::P) sm[l * S::LS + pad(S::P - k)] = make_float2(v.x + v.w, v.z - v.y);
            }
        }
    }
    __syncthreads();
    fft_x_lines<LOGP, R0, S::NL, true>(sm, p.tw, p.twr[R0]);
    const int cur = s_cur;
    const float* min = src_ptr(p, a.src, cur);
    Partials pt = {0.f, 0.f, 0.0, 0.0, 0u};
    const StageCoefs& sc = s_sc;
    const int NX = p.nx, NY = p.ny;
    // one item = one x and a pair of rows (2q, 2q+1): component c of that pair
    // is the complex entry (line c*TY/2 + q, position x)
    for (int idx = threadIdx.x; idx < HP * NX; idx += S::NT) {
        const int q = idx / NX, x = idx - q * NX;
        const int y = y0 + 2 * q;
        float2* e0 = sm + (0 * HP + q) * S::LS + pad(x);
        float2* e1 = sm + (1 * HP + q) * S::LS + pad(x);
        float2* e2 = sm + (2 * HP + q) * S::LS + pad(x);
        const float2 h0 = *e0, h1 = *e1, h2 = *e2;
        f3 na = mk(0.f, 0.f, 0.f), nb = mk(0.f, 0.f, 0.f);
        const long long cell = ((long long)z * NY + y) * NX + x;
        if (y < NY) na = cell_update<LITE>(p, a, cur, sc, min, cell, x, y, z, mk(h0.x, h1.x, h2.x), s_tstep, pt);
        if (y + 1 < NY)
            nb = cell_update<LITE>(p, a, cur, sc, min, cell + NX, x, y + 1, z, mk(h0.y, h1.y, h2.y), s_tstep, pt);
        if constexpr (FUSE) {
            *e0 = make_float2(na.x, nb.x);
            *e1 = make_float2(na.y, nb.y);
            *e2 = make_float2(na.z, nb.z);
        }
    }
    if constexpr (FUSE) {
        // zero padding of the next transform: x in [nx, P)
        const int W = S::P - NX;
        for (int idx = threadIdx.x; idx < S::NL * W; idx += S::NT) {
            const int l = idx / W, x = NX + (idx - l * W);
            sm[l * S::LS + pad(x)] = make_float2(0.f, 0.f);
        }
        __syncthreads();
        fft_x_lines<LOGP, R0, S::NL, false>(sm, p.tw, p.twr[R0]);
        store_x_spectrum<LOGP, R0>(p, sm, y0, z);
    }
    reduce_and_finish(p, a, pt, gridDim.x * gridDim.y);
}

// ---------------------------------------------------------------------------
// x passes in the register style of the column pass (P >= 64).  A block holds
// PAIRS row pairs; each thread owns the same radix-8 butterflies of the three
// component lines of one pair (a complex line packs rows y and y+1), so the
// twiddles are shared and every pass has three independent butterflies in
// flight.  The inverse transform's first pass reads the half spectrum from
// global memory directly (unpacking each row pair's two real spectra into one
// complex line), and the forward transform of the next evaluation's input
// starts from the epilogue's output.
// FFT lengths the batched passes are compiled for: 2^6..2^10 along x and y,
// 2^1..2^10 along z
constexpr int BATCH_MIN_LOGP = 6, BATCH_MAX_LOGP = 10;
#ifndef XR_MINB256
#define XR_MINB256 3
#endif

// HALF = 1: half the row pairs per block (a tile shape the batch autotuner
// times against the default)
template <int LOGP, int HALF = 0>
struct XR {
    using PL = r8::Plan8<LOGP>;
    static constexpr int P = PL::P, NB = PL::NB, LS = PL::LS;
    static constexpr int PAIRS0 = NB >= 256 ? 1 : (256 / NB > 8 ? 8 : 256 / NB);
    static constexpr int PAIRS = HALF && PAIRS0 > 1 ? PAIRS0 / 2 : PAIRS0;
    static constexpr int TY = 2 * PAIRS;
    static constexpr int NT = (PAIRS * NB + 31) / 32 * 32 < 64 ? 64 : (PAIRS * NB + 31) / 32 * 32;
    static constexpr int HX = P / 2 + 1;
    static constexpr int NL = 3 * PAIRS;
    static constexpr int LASTF = PL::NPASS - 1;
    static constexpr int MINB = NT >= 256 ? XR_MINB256 : 1024 / NT;
    static constexpr int MINB1 = NT >= 256 ? XR_MINB256 : 65536 / (NT * 80);   // >= 80 registers (autotuner)
    static constexpr size_t SMEM = (size_t)NL * LS * sizeof(float2);
};

// Unpack of the paired rows (A = (Z_k + conj Z_-k)/2, B = (Z_k - conj Z_-k)/(2i))
// and transposed store to s1 [c][kx][z][y] for lines laid out as
// line (c, q) = sm + (c*PAIRS + q)*LS, q the row pair.
template <int LOGP, int HALF = 0>
__device__ __forceinline__ void store_x_spectrum_r(const HotParams& p, const float2* sm, int y0, int z) {
    using S = XR<LOGP, HALF>;
    for (int idx = threadIdx.x; idx < S::NL * S::HX; idx += S::NT) {
        const int l = idx / S::HX, k = idx - l * S::HX;
        const float2 A = sm[l * S::LS + pad(k)];
        const float2 B = cconj(sm[l * S::LS + pad((S::P - k) & (S::P - 1))]);
        const float2 D = csub(A, B);
        const float4 out = make_float4(0.5f * (A.x + B.x), 0.5f * (A.y + B.y), 0.5f * D.y, -0.5f * D.x);
        const int c = l / S::PAIRS, q = l - c * S::PAIRS;
        float2* dst = p.s1 + ((long long)(c * S::HX + k) * p.nz + z) * p.nyp + y0 + 2 * q;
        *reinterpret_cast<float4*>(dst) = out;
    }
}

// forward transform of the lines whose pass-0 inputs are in v (REV = false
// order) and transposed store of the half spectrum
template <int LOGP, int HALF = 0>
__device__ __forceinline__ void xr_forward_store(const HotParams& p, float2* const* lines, float2 (*v)[8], int j,
                                                 bool act, bool from_smem, int y0, int z, float2* sm) {
    using S = XR<LOGP, HALF>;
    r8::run<LOGP, false, false, 0, 3>(lines, v, j, act, p.tw, from_smem);
    __syncthreads();
    if (act) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < 8; ++i) lines[c][pad(r8::out_pos<LOGP, false, S::LASTF>(j, i))] = v[c][i];
    }
    __syncthreads();
    store_x_spectrum_r<LOGP, HALF>(p, sm, y0, z);
}

template <int LOGP, int HALF = 0>
__device__ __forceinline__ void xfwd_r_body(const HotParams& p, const LaunchArgs& a, int bx, int by) {
    using S = XR<LOGP, HALF>;
    extern __shared__ float2 sm[];
    const int y0 = bx * S::TY, z = by;
    DevState* st = p.st;
    if (!a.keep && a.mode != LM_EVAL && st->done) return;
    const int cur = st->cur;
    const long long n = p.ncell;
    const bool comb = a.src == SRC_COMBINE2;
    const float* src = comb ? p.ms[cur] : src_ptr(p, a.src, cur);
    const float* k1 = p.ks[cur];
    float* wout = p.mstage[0];
    const Coef c21 = comb ? split(st->h * c_rka[p.rk][2][1]) : Coef{0.f, 0.f};
    const int NX = p.nx, NY = p.ny;
    const int tid = threadIdx.x;
    int q = tid / S::NB;
    const int j = tid - q * S::NB;
    const bool act = q < S::PAIRS;
    if (!act) q = 0;
    float2* lines[3] = {sm + (0 * S::PAIRS + q) * S::LS, sm + (1 * S::PAIRS + q) * S::LS,
                        sm + (2 * S::PAIRS + q) * S::LS};
    const int y = y0 + 2 * q;
    float2 v[3][8];
    if (act) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int x = r8::in_pos<LOGP, false, 0>(j, i);
                float2 w = make_float2(0.f, 0.f);
                if (x < NX) {
                    const long long i0 = (long long)c * n + ((long long)z * NY + y) * NX + x;
                    if (y < NY) {
                        float u = src[i0];
                        if (comb) { u = fmaf(c21.lo, k1[i0], fmaf(c21.hi, k1[i0], u)); wout[i0] = u; }
                        w.x = u;
                    }
                    if (y + 1 < NY) {
                        float u = src[i0 + NX];
                        if (comb) { u = fmaf(c21.lo, k1[i0 + NX], fmaf(c21.hi, k1[i0 + NX], u)); wout[i0 + NX] = u; }
                        w.y = u;
                    }
                }
                v[c][i] = w;
            }
    }
    xr_forward_store<LOGP, HALF>(p, lines, v, j, act, false, y0, z, sm);
}

template <int LOGP>
__global__ void __launch_bounds__(XR<LOGP>::NT, XR<LOGP>::MINB) k_xfwd_r(HotParams p, LaunchArgs a) {
    xfwd_r_body<LOGP>(p, a, blockIdx.x, blockIdx.y);
}
// V: 0 the default budget, 1 at least 80 registers, 2 half the row pairs per block
template <int LOGP, int V>
__global__ void __launch_bounds__(XR<LOGP, V == 2>::NT, V == 1 ? XR<LOGP>::MINB1 : XR<LOGP, V == 2>::MINB)
kb_xfwd_r(const HotParams* __restrict__ ps, const int4* __restrict__ work, LaunchArgs a) {
    const int4 w = work[blockIdx.x];
    __shared__ HotParams s_hp;
    load_params(ps + w.x, &s_hp);
    xfwd_r_body<LOGP, V == 2>(s_hp, a, w.y, w.z);
}

// Inverse x pass alone (C2R + crop): H_demag into hbuf [3][ncell], stored
// straight from the registers of the last pass (thread j holds positions
// j + r*P/8, so a warp stores consecutive x).
template <int LOGP, int HALF = 0>
__device__ __forceinline__ void xinv_h_body(const HotParams& p, const LaunchArgs& a, int bx, int by) {
    using S = XR<LOGP, HALF>;
    extern __shared__ float2 sm[];
    const int y0 = bx * S::TY, z = by;
    if (a.mode != LM_EVAL && p.st->done) return;
    const int tid = threadIdx.x;
    int q = tid / S::NB;
    const int j = tid - q * S::NB;
    const bool act = q < S::PAIRS;
    if (!act) q = 0;
    float2* lines[3] = {sm + (0 * S::PAIRS + q) * S::LS, sm + (1 * S::PAIRS + q) * S::LS,
                        sm + (2 * S::PAIRS + q) * S::LS};
    float2 v[3][8];
    if (act) {
        const long long cs = (long long)S::HX * p.nz * p.nyp;
        const float2* base = p.s1 + (long long)z * p.nyp + y0 + 2 * q;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int pos = r8::in_pos<LOGP, true, 0>(j, i);
            const bool mir = pos > (S::P >> 1);
            const int k = mir ? S::P - pos : pos;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                // (A, B) = the two rows' spectra at k; Z = A + iB, Z[-k] = conj A + i conj B
                const float4 w = __ldg(reinterpret_cast<const float4*>(base + c * cs + (long long)k * p.nz * p.nyp));
                v[c][i] = mir ? make_float2(w.x + w.w, w.z - w.y) : make_float2(w.x - w.w, w.y + w.z);
            }
        }
    }
    r8::run<LOGP, true, true, 0, 3>(lines, v, j, act, p.tw, false);
    if (act) {
        const int NX = p.nx, NY = p.ny, y = y0 + 2 * q;
        const long long n = p.ncell;
        const long long row = ((long long)z * NY + y) * NX;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int x = r8::out_pos<LOGP, true, S::LASTF>(j, i);
            if (x < NX) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (y < NY) p.hbuf[c * n + row + x] = v[c][i].x;
                    if (y + 1 < NY) p.hbuf[c * n + row + NX + x] = v[c][i].y;
                }
            }
        }
    }
}

template <int LOGP>
__global__ void __launch_bounds__(XR<LOGP>::NT, XR<LOGP>::MINB) k_xinv_h(HotParams p, LaunchArgs a) {
    xinv_h_body<LOGP>(p, a, blockIdx.x, blockIdx.y);
}
template <int LOGP, int V>
__global__ void __launch_bounds__(XR<LOGP, V == 2>::NT, V == 1 ? XR<LOGP>::MINB1 : XR<LOGP, V == 2>::MINB)
kb_xinv_h(const HotParams* __restrict__ ps, const int4* __restrict__ work, LaunchArgs a) {
    const int4 w = work[blockIdx.x];
    __shared__ HotParams s_hp;
    load_params(ps + w.x, &s_hp);
    xinv_h_body<LOGP, V == 2>(s_hp, a, w.y, w.z);
}

// Cell pass: local terms, torque and stage update for every cell, with the
// magnetostatic field from hbuf when demag is on (the inverse x pass wrote
// it) and without it otherwise.
template <bool EV>
__device__ __forceinline__ void local_body(const HotParams& p, const LaunchArgs& a, int bx, int nblk) {
    __shared__ StageCoefs s_sc;
    __shared__ long long s_tstep;
    DevState* st = p.st;
    if (a.mode != LM_EVAL && st->done) return;
    // the first warp forms the stage weights while every thread issues its loads
    if (threadIdx.x < 32) stage_coefs(p, a, st, s_sc);
    if (threadIdx.x == 0) s_tstep = (a.mode == LM_EVAL) ? p.thermal_step : st->step_index;
    const int cur = st->cur;
    const float* min = src_ptr(p, a.src, cur);
    const long long n = p.ncell;
    const long long cell = bx * 256ll + threadIdx.x;
    const bool valid = cell < n;
    const int NX = p.nx, NY = p.ny;
    int x = 0, y = 0, z = 0;
    if (valid) {
        if (n <= 0xffffffffll) {                   // 32-bit division where it suffices
            const unsigned c32 = (unsigned)cell, r = c32 / (unsigned)NX;
            x = (int)(c32 - r * (unsigned)NX);
            y = (int)(r % (unsigned)NY);
            z = (int)(r / (unsigned)NY);
        } else {
            const long long r = cell / NX;
            x = (int)(cell - r * NX);
            y = (int)(r % NY);
            z = (int)(r / NY);
        }
    }
    CellIn in;
    f3 hd = mk(0.f, 0.f, 0.f);
    if (valid) {
        load_cell(p, a, cur, min, cell, x, y, z, in);
        if (p.demag) hd = ld3(p.hbuf, cell, n);
    }
    __syncthreads();
    Partials pt = {0.f, 0.f, 0.0, 0.0, 0u};
    if (valid) update_cell<EV>(p, a, cur, s_sc, cell, in, hd, s_tstep, pt);
    reduce_and_finish<EV>(p, a, pt, nblk);
}

// the LITE fused x kernels cover padded x lengths of 64 and more (measured on
// the 1024^2 film: 73.5 against 79.1 us per fused launch, no spills against
// 64 bytes; with three blocks per SM instead of two, 56 registers and 148
// bytes of spills, it took 80 us)
constexpr int LITE_MIN_LOGP = 6;
static bool lite_terms(const HotParams& p) {
    return p.nz == 1 && !p.pbc[2] && !p.uaxis && p.kc1 == 0.f && p.kc2 == 0.f && !(p.sigma_th > 0.f) && !p.stt;
}

// ---------------------------------------------------------------------------
// launch helpers

}  // namespace mm
