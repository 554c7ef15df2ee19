// hotpath_small.cu - a whole field evaluation of a small 2-D grid in ONE launch:
// one thread-block cluster whose CTAs keep the half spectrum in their shared
// memory (distributed shared memory), so the x forward pass, the y column pass
// with the kernel product, the x inverse pass and the cell terms of Sec. 3.2
// run back to back without a trip through HBM or a kernel boundary.
//
// Layout.  CTA r of the cluster owns the kx columns [r HC, (r + 1) HC) of the
// half spectrum, SP_r[c][kx - r HC][y] (y < ny rounded up to even, complex),
// and the row pairs [q0_r, q1_r) of the grid.  The x passes transform two real
// rows of a component as one complex line (as the multi-kernel passes do) and
// store bin k of both rows into the owner of column k (a 16-byte remote store);
// the column pass runs on the CTA's own columns; the inverse x pass reads its
// row pairs' bins back from the owners.  Four cluster barriers order the
// phases: after start-up (every CTA's shared memory exists before any remote
// store), after the x forward pass, after the column pass, and after the last
// remote read (no CTA leaves while another still reads its shared memory).
// The reductions and the step control are those of the multi-kernel passes
// (reduce_and_finish over the cluster's CTAs).
//
// The 1-D transforms are radix-8 Stockham passes (then one radix-4 or radix-2
// pass for the rest of log2 P) over lines in shared memory, with the line
// length a run-time value, so one kernel serves every length; the twiddles
// are copied into shared memory once per evaluation.  A run of steps can be
// one launch (k_small_steps): the evaluations of each standard step in turn,
// a cluster barrier after each one's step control.
#include "hotpath_kernels.cuh"

#include <cooperative_groups.h>

namespace mm {
namespace cg = cooperative_groups;

namespace {

constexpr int SMALL_NT = 512;          // threads per CTA
constexpr int SMALL_PTS = 4096;        // complex points per transform call (all lines)
constexpr int SMALL_MAX_CL = 16;       // CTAs per cluster (16: the non-portable size)
constexpr size_t SMALL_MAX_SMEM = 200 * 1024;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
// 4- and 8-byte asynchronous global -> shared copies; nbytes = 0 fills zeros
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int nbytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(nbytes));
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// One radix-R pass (R = 8, 4 or 2) of a Stockham transform over nl lines of
// length P = 2^logp at base + l * ls (padded index pad()); ns = product of the
// radices before this pass; tab[t] = exp(-2 pi i t / P) in shared memory,
// conjugated for the inverse.  Every thread calls it; each owns at most
// SMALL_PTS / (SMALL_NT R) butterflies.
template <int R>
__device__ __forceinline__ void rt_pass(float2* base, int ls, int nl, int logp, int ns, const float2* tab, bool inv) {
    using namespace mmfft;
    constexpr int IPT = SMALL_PTS / (SMALL_NT * R);
    constexpr int LR = R == 8 ? 3 : R == 4 ? 2 : 1;
    const int lognb = logp - LR, nb = 1 << lognb;
    const int items = nl << lognb;
    const int tstep = (1 << logp) / (ns * R);      // twiddle index unit of this pass
    float2 v[IPT][R];
#pragma unroll
    for (int t = 0; t < IPT; ++t) {
        const int it = threadIdx.x + t * SMALL_NT;
        if (it < items) {
            const int l = it >> lognb, j = it & (nb - 1);
            const float2* a = base + l * ls;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 x = a[pad(j + r * nb)];
                v[t][r] = inv ? cconj(x) : x;          // inverse = conj(forward(conj))
            }
            if (ns > 1) {
                const int t1 = (j & (ns - 1)) * tstep;
#pragma unroll
                for (int r = 1; r < R; ++r) v[t][r] = cmul(v[t][r], tab[r * t1]);
            }
            dft<R, false>(v[t]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < IPT; ++t) {
        const int it = threadIdx.x + t * SMALL_NT;
        if (it < items) {
            const int l = it >> lognb, j = it & (nb - 1);
            const int k = j & (ns - 1), o = (j - k) * R + k;
            float2* a = base + l * ls;
#pragma unroll
            for (int r = 0; r < R; ++r) a[pad(o + r * ns)] = inv ? cconj(v[t][r]) : v[t][r];
        }
    }
    __syncthreads();
}

// In-place FFT (no 1/P scaling) of nl lines of length 2^logp, nl 2^logp <=
// SMALL_PTS: radix-8 passes, then one radix-4 or radix-2 pass for the rest;
// inv: the inverse transform.  Called by every thread after the lines are
// written; ends with a barrier.  One copy of the code serves all four
// transforms of an evaluation (the kernel is bound by instruction fetch).
__device__ __noinline__ void fft_rt(float2* base, int ls, int nl, int logp, const float2* tab, bool inv) {
    int ns = 1, rem = logp;
    while (rem >= 3) {
        rt_pass<8>(base, ls, nl, logp, ns, tab, inv);
        ns <<= 3;
        rem -= 3;
    }
    if (rem == 2) rt_pass<4>(base, ls, nl, logp, ns, tab, inv);
    else if (rem == 1) rt_pass<2>(base, ls, nl, logp, ns, tab, inv);
}

}  // namespace

// Shape of the one-launch evaluation (host and device compute it alike).
struct SmallShape {
    int cl;             // CTAs in the cluster
    int hx, hc;         // half-spectrum columns; columns per CTA
    int nye, nq;        // rows rounded up to even; row pairs
    int qc, cc;         // row pairs per x-transform call; columns per column call
    int lsx, lsy;       // padded line strides
    int hyk;            // kernel entries per column (py/2 + 1)
    int sp, wk, kt;     // float2 elements of the spectrum slice, the work lines and the kernel slice
    int total;          // float2 elements in all, with the twiddle tables (px + py)
};

__host__ __device__ inline SmallShape small_shape(int nx, int ny, int logpx, int logpy, int cl) {
    (void)nx;
    SmallShape s;
    const int px = 1 << logpx, py = 1 << logpy;
    s.cl = cl;
    s.hx = px / 2 + 1;
    s.hc = (s.hx + cl - 1) / cl;
    s.nye = (ny + 1) & ~1;
    s.nq = s.nye / 2;
    s.lsx = mmfft::padded_len(px);
    s.lsy = mmfft::padded_len(py);
    const int qmax = SMALL_PTS / (3 * px);
    const int qper = (s.nq + cl - 1) / cl;
    s.qc = qmax < 1 ? 1 : (qmax < qper ? qmax : qper);
    const int cmax = SMALL_PTS / (3 * py);
    s.cc = cmax < 1 ? 1 : (cmax < s.hc ? cmax : s.hc);
    s.hyk = py / 2 + 1;
    s.sp = 3 * s.hc * s.nye;
    s.sp = (s.sp + 1) & ~1;                     // every region starts 16-byte aligned
    const int wx = 3 * s.qc * s.lsx, wy = 3 * s.cc * s.lsy;
    s.wk = ((wx > wy ? wx : wy) + 1) & ~1;
    s.kt = (4 * s.cc * s.hyk + 3) / 4 * 2;      // 4 kernel components as floats, in float2 units
    s.total = s.sp + s.wk + s.kt + px + py;
    return s;
}

// One evaluation (every thread of every CTA of the cluster calls it).  Returns
// false without doing anything when the run has already finished; that
// answer is the same in every CTA: nothing writes the device state's done
// flag between the evaluation's start and its last CTA's step control.
// LITE: the film's term set (one easy axis, no cubic anisotropy, thermal field
// or spin-transfer torque), compiled without the other terms' code.
template <bool LITE>
__device__ __forceinline__ bool small_eval(const HotParams& p, const LaunchArgs& a, const SmallShape& S,
                                           float2* smem) {
    using namespace mmfft;
    __shared__ StageCoefs s_sc;
    __shared__ int s_cur, s_done;
    __shared__ long long s_tstep;
    __shared__ Coef s_c21;
    __shared__ DevState s_st;                        // the fields stage_coefs reads (h)
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    if (tid == 0) {
        // volatile: in a persistent launch another CTA's step control wrote these
        // since this SM last read them; read them from L2, never from L1
        const volatile DevState* vs = p.st;
        s_done = (a.mode != LM_EVAL && vs->done) ? 1 : 0;
        s_cur = vs->cur;
        s_tstep = (a.mode == LM_EVAL) ? p.thermal_step : vs->step_index;
        s_st.h = vs->h;
        s_c21 = a.src == SRC_COMBINE2 ? split(s_st.h * c_rka[p.rk][2][1]) : Coef{0.f, 0.f};
    }
    __syncthreads();
    if (tid < 32) stage_coefs(p, a, &s_st, s_sc);
    __syncthreads();
    if (s_done) return false;                        // the whole cluster returns here
    cluster.sync();                                  // (1) every CTA's shared memory exists (and
                                                     // the previous evaluation's reads of it are over)

    float2* SP = smem;                               // this CTA's spectrum columns
    float2* WK = SP + S.sp;                          // work lines
    float* KT = reinterpret_cast<float*>(WK + S.wk); // kernel slice of a column chunk
    float2* TWX = WK + S.wk + S.kt;                  // exp(-2 pi i t / Px), t < Px
    float2* TWY = TWX + p.px;                        // exp(-2 pi i t / Py), t < Py
    const int NX = p.nx, NY = p.ny, PX = p.px, PY = p.py;
    const int HX = S.hx, HC = S.hc, NYE = S.nye;
    const int cur = s_cur;
    const long long n = p.ncell;
    const int q0 = (int)((long long)rank * S.nq / S.cl), q1 = (int)((long long)(rank + 1) * S.nq / S.cl);
    const int kx0 = rank * HC, kx1 = kx0 + HC < HX ? kx0 + HC : HX;
    // the twiddles of both lengths, from the table of exp(-2 pi i t / TWN)
    for (int t = tid; t < PX + PY; t += SMALL_NT) {
        const int tx = t < PX ? t * (TWN >> p.logpx) : (t - PX) * (TWN >> p.logpy);
        cp_async8(TWX + t, p.tw + tx);
    }

    // ---- x forward: rows of the evaluation input -> bins to their owners ----
    {
        const bool comb = a.src == SRC_COMBINE2;
        const float* src = comb ? p.ms[cur] : src_ptr(p, a.src, cur);
        const float* k1 = p.ks[cur];
        float* wout = p.mstage[0];
        const Coef c21 = s_c21;
        for (int qa = q0; qa < q1; qa += S.qc) {
            const int qn = q1 - qa < S.qc ? q1 - qa : S.qc, nl = 3 * qn;
            if (!comb) {
                // rows y and y + 1 of a component as the real and imaginary parts of one line,
                // zero past the grid: asynchronous copies, all in flight at once
                for (int idx = tid; idx < nl * PX; idx += SMALL_NT) {
                    const int l = idx >> p.logpx, x = idx & (PX - 1);
                    const int c = l / qn, y = 2 * (qa + (l - c * qn));
                    const long long i0 = (long long)c * n + (long long)y * NX + x;
                    float* d = reinterpret_cast<float*>(WK + l * S.lsx + pad(x));
                    const bool in0 = x < NX && y < NY, in1 = x < NX && y + 1 < NY;
                    cp_async4(d, in0 ? src + i0 : src, in0 ? 4 : 0);
                    cp_async4(d + 1, in1 ? src + i0 + NX : src, in1 ? 4 : 0);
                }
                cp_async_wait_all();
            } else {
                // stage-2 input m_n + h a21 k1 (also written to mstage[0]): four items' loads in flight
                for (int i0w = 0; i0w < nl * PX; i0w += 4 * SMALL_NT) {
                    float u0[4], u1[4], g0[4], g1[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int idx = i0w + tid + q * SMALL_NT;
                        u0[q] = u1[q] = g0[q] = g1[q] = 0.f;
                        if (idx < nl * PX) {
                            const int l = idx >> p.logpx, x = idx & (PX - 1);
                            const int c = l / qn, y = 2 * (qa + (l - c * qn));
                            const long long i0 = (long long)c * n + (long long)y * NX + x;
                            if (x < NX && y < NY) { u0[q] = src[i0]; g0[q] = k1[i0]; }
                            if (x < NX && y + 1 < NY) { u1[q] = src[i0 + NX]; g1[q] = k1[i0 + NX]; }
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int idx = i0w + tid + q * SMALL_NT;
                        if (idx < nl * PX) {
                            const int l = idx >> p.logpx, x = idx & (PX - 1);
                            const int c = l / qn, y = 2 * (qa + (l - c * qn));
                            const long long i0 = (long long)c * n + (long long)y * NX + x;
                            float2 v = make_float2(0.f, 0.f);
                            if (x < NX && y < NY) { v.x = fmaf(c21.lo, g0[q], fmaf(c21.hi, g0[q], u0[q])); wout[i0] = v.x; }
                            if (x < NX && y + 1 < NY) {
                                v.y = fmaf(c21.lo, g1[q], fmaf(c21.hi, g1[q], u1[q]));
                                wout[i0 + NX] = v.y;
                            }
                            WK[l * S.lsx + pad(x)] = v;
                        }
                    }
                }
                cp_async_wait_all();                 // the twiddle tables
            }
            __syncthreads();
            fft_rt(WK, S.lsx, nl, p.logpx, TWX, false);
            for (int idx = tid; idx < nl * HX; idx += SMALL_NT) {
                const int l = idx / HX, k = idx - l * HX;
                const int c = l / qn, y = 2 * (qa + (l - c * qn));
                // two real rows in one line: A_k = (Z_k + conj Z_-k)/2, B_k = (Z_k - conj Z_-k)/(2i)
                const float2 A = WK[l * S.lsx + pad(k)];
                const float2 Bc = cconj(WK[l * S.lsx + pad(k == 0 ? 0 : PX - k)]);
                const float2 D = csub(A, Bc);
                const int own = k / HC;
                float2* dst = cluster.map_shared_rank(SP, own) + (c * HC + (k - own * HC)) * NYE + y;
                *reinterpret_cast<float4*>(dst) =
                    make_float4(0.5f * (A.x + Bc.x), 0.5f * (A.y + Bc.y), 0.5f * D.y, -0.5f * D.x);
            }
            __syncthreads();
        }
        cp_async_wait_all();                         // a CTA without rows still has the tables
        __syncthreads();
    }
    cluster.sync();                                  // (2) every bin is with its owner

    // ---- column pass on the own columns: FFT along y, kernel product, inverse ----
    {
        const long long cs = (long long)HX * p.hyk * p.hzk;
        const int HYK = S.hyk;
        for (int ka = kx0; ka < kx1; ka += S.cc) {
            const int cn = kx1 - ka < S.cc ? kx1 - ka : S.cc, nl = 3 * cn;
            // the chunk's kernel columns (4 components, kq = 0..Py/2 each), copied
            // while the forward transform runs
            for (int idx = tid; idx < 4 * cn * HYK; idx += SMALL_NT) {
                const int comp = idx / (cn * HYK), r = idx - comp * (cn * HYK);
                cp_async4(KT + idx, p.kt + comp * cs + (long long)ka * HYK + r, 4);
            }
            for (int idx = tid; idx < nl * PY; idx += SMALL_NT) {
                const int l = idx >> p.logpy, y = idx & (PY - 1);
                const int c = l / cn, kl = ka - kx0 + (l - c * cn);
                WK[l * S.lsy + pad(y)] = y < NY ? SP[(c * HC + kl) * NYE + y] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            fft_rt(WK, S.lsy, nl, p.logpy, TWY, false);
            cp_async_wait_all();
            __syncthreads();
            for (int idx = tid; idx < cn * PY; idx += SMALL_NT) {
                const int cc = idx >> p.logpy, pos = idx & (PY - 1);
                const bool hi = pos > (PY >> 1);
                const int kq = hi ? PY - pos : pos;
                const int b = cc * HYK + kq, cs4 = cn * HYK;
                const float kxx = KT[b], kyy = KT[cs4 + b], kzz = KT[2 * cs4 + b];
                const float kxy = hi ? -KT[3 * cs4 + b] : KT[3 * cs4 + b];
                float2* e0 = WK + (0 * cn + cc) * S.lsy + pad(pos);
                float2* e1 = WK + (1 * cn + cc) * S.lsy + pad(pos);
                float2* e2 = WK + (2 * cn + cc) * S.lsy + pad(pos);
                const float2 X = *e0, Y = *e1, Z = *e2;
                *e0 = make_float2(kxx * X.x + kxy * Y.x, kxx * X.y + kxy * Y.y);
                *e1 = make_float2(kxy * X.x + kyy * Y.x, kxy * X.y + kyy * Y.y);
                *e2 = make_float2(kzz * Z.x, kzz * Z.y);
            }
            __syncthreads();
            fft_rt(WK, S.lsy, nl, p.logpy, TWY, true);
            for (int idx = tid; idx < nl * NY; idx += SMALL_NT) {
                const int l = idx / NY, y = idx - l * NY;
                const int c = l / cn, kl = ka - kx0 + (l - c * cn);
                SP[(c * HC + kl) * NYE + y] = WK[l * S.lsy + pad(y)];
            }
            __syncthreads();
        }
    }
    cluster.sync();                                  // (3) every column is transformed

    // ---- x inverse + crop + cell terms of the own rows ----
    Partials pt = {0.f, 0.f, 0.0, 0.0, 0u};
    {
        const float* min = src_ptr(p, a.src, cur);
        const StageCoefs& sc = s_sc;
        const long long tstep = s_tstep;
        for (int qa = q0; qa < q1; qa += S.qc) {
            const int qn = q1 - qa < S.qc ? q1 - qa : S.qc, nl = 3 * qn;
            for (int idx = tid; idx < nl * HX; idx += SMALL_NT) {
                const int l = idx / HX, k = idx - l * HX;
                const int c = l / qn, y = 2 * (qa + (l - c * qn));
                const int own = k / HC;
                const float4 v = *reinterpret_cast<const float4*>(
                    cluster.map_shared_rank(SP, own) + (c * HC + (k - own * HC)) * NYE + y);
                // Z = A + iB with A = (v.x, v.y), B = (v.z, v.w); Z[-k] = conj(A) + i conj(B)
                WK[l * S.lsx + pad(k)] = make_float2(v.x - v.w, v.y + v.z);
                if (k > 0 && 2 * k < PX) WK[l * S.lsx + pad(PX - k)] = make_float2(v.x + v.w, v.z - v.y);
            }
            __syncthreads();
            fft_rt(WK, S.lsx, nl, p.logpx, TWX, true);
            for (int idx = tid; idx < qn * NX; idx += SMALL_NT) {
                const int qq = idx / NX, x = idx - qq * NX;
                const int y = 2 * (qa + qq);
                const float2 h0 = WK[(0 * qn + qq) * S.lsx + pad(x)];
                const float2 h1 = WK[(1 * qn + qq) * S.lsx + pad(x)];
                const float2 h2 = WK[(2 * qn + qq) * S.lsx + pad(x)];
                const long long cell = (long long)y * NX + x;
                if (y < NY) cell_update<LITE>(p, a, cur, sc, min, cell, x, y, 0, mk(h0.x, h1.x, h2.x), tstep, pt);
                if (y + 1 < NY)
                    cell_update<LITE>(p, a, cur, sc, min, cell + NX, x, y + 1, 0, mk(h0.y, h1.y, h2.y), tstep, pt);
            }
            __syncthreads();
        }
    }
    cluster.sync();                                  // (4) no remote read is left
    reduce_and_finish(p, a, pt, S.cl);
    return true;
}

template <bool LITE>
__global__ void __launch_bounds__(SMALL_NT, 1) k_small(HotParams p, LaunchArgs a, SmallShape S) {
    extern __shared__ __align__(16) float2 smem[];
    small_eval<LITE>(p, a, S, smem);
}

// The standard step's evaluations, nsteps times, in one launch: the code stays
// in the instruction cache from one evaluation to the next.  After each
// evaluation a cluster barrier waits for its step control (run in the last CTA
// to finish it) so that the next one reads the updated device state.
template <bool LITE>
__global__ void __launch_bounds__(SMALL_NT, 1) k_small_steps(HotParams p, SmallSteps L, SmallShape S) {
    extern __shared__ __align__(16) float2 smem[];
    cg::cluster_group cluster = cg::this_cluster();
    for (long long step = 0; step < L.nsteps; ++step) {
        for (int e = 0; e < L.n; ++e) {
            if (!small_eval<LITE>(p, L.a[e], S, smem)) return;     // finished: the same answer in every CTA
            __threadfence();
            cluster.sync();
            __threadfence();                         // the step control's writes before any read of them
        }
    }
}

// the largest cluster this device co-schedules with the kernel's shared
// memory (set by configure_small_kernels)
static int g_small_max_cl = 0;

// CTAs per cluster for a context, 0 when the one-launch evaluation does not
// apply: 2-D (nz = 1, open z), power-of-two lengths along x and y, and a
// spectrum slice plus work lines that fit one CTA's shared memory.  The
// smallest cluster that fits is taken, at least one CTA per 1024 cells.
int small_cluster_size(const HotParams& p) {
    if (p.nz != 1 || p.pbc[2] || p.rx != 1 || p.ry != 1) return 0;
    if (p.logpx < 1 || p.logpx > 10 || p.logpy > 10) return 0;
    if (3 * (1 << p.logpx) > SMALL_PTS || 3 * (1 << p.logpy) > SMALL_PTS) return 0;
    const int maxcl = g_small_max_cl > 0 ? g_small_max_cl : SMALL_MAX_CL;
    long long want = (p.ncell + 1023) / 1024;
    for (int cl = 1; cl <= maxcl; cl *= 2) {
        if (cl < want && cl < maxcl) continue;
        const SmallShape s = small_shape(p.nx, p.ny, p.logpx, p.logpy, cl);
        if ((size_t)s.total * sizeof(float2) <= SMALL_MAX_SMEM) return cl;
    }
    return 0;
}

// launch configuration of one cluster of p.small_cl CTAs; false if it does not apply
static bool small_config(const HotParams& p, cudaStream_t s, SmallShape* S, cudaLaunchConfig_t* cfg,
                         cudaLaunchAttribute* attr) {
    const int cl = p.small_cl;
    if (cl < 1 || cl > SMALL_MAX_CL) return false;
    *S = small_shape(p.nx, p.ny, p.logpx, p.logpy, cl);
    const size_t smem = (size_t)S->total * sizeof(float2);
    if (smem > SMALL_MAX_SMEM) return false;
    *cfg = cudaLaunchConfig_t{};
    cfg->gridDim = dim3(cl, 1, 1);
    cfg->blockDim = dim3(SMALL_NT, 1, 1);
    cfg->dynamicSmemBytes = smem;
    cfg->stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg->attrs = attr;
    cfg->numAttrs = 1;
    return true;
}

cudaError_t launch_small(const HotParams& p, const LaunchArgs& a, cudaStream_t s) {
    SmallShape S;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    if (!small_config(p, s, &S, &cfg, attr)) return cudaErrorInvalidValue;
    if (lite_terms(p)) return cudaLaunchKernelEx(&cfg, k_small<true>, p, a, S);
    return cudaLaunchKernelEx(&cfg, k_small<false>, p, a, S);
}

cudaError_t launch_small_steps(const HotParams& p, const SmallSteps& steps, cudaStream_t s) {
    SmallShape S;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    if (!small_config(p, s, &S, &cfg, attr) || steps.n < 1 || steps.n > 8 || steps.nsteps < 1)
        return cudaErrorInvalidValue;
    if (lite_terms(p)) return cudaLaunchKernelEx(&cfg, k_small_steps<true>, p, steps, S);
    return cudaLaunchKernelEx(&cfg, k_small_steps<false>, p, steps, S);
}

cudaError_t configure_small_kernels() {
    cudaError_t e;
    for (auto k : {k_small<false>, k_small<true>}) {
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMALL_MAX_SMEM))) return e;
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1))) return e;
    }
    for (auto k : {k_small_steps<false>, k_small_steps<true>}) {
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMALL_MAX_SMEM))) return e;
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1))) return e;
    }
    // largest power-of-two cluster that can be resident with the full shared memory
    int best = 0;
    for (int cl = 1; cl <= SMALL_MAX_CL; cl *= 2) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cl, 1, 1);
        cfg.blockDim = dim3(SMALL_NT, 1, 1);
        cfg.dynamicSmemBytes = SMALL_MAX_SMEM;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_small<false>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            break;
        }
        if (n < 1) break;
        best = cl;
    }
    g_small_max_cl = best > 0 ? best : 1;
    return cudaSuccess;
}

}  // namespace mm
