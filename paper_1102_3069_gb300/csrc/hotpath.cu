// hotpath.cu - the passes of the effective field and the time step: the
// power-of-two lengths, the cell passes, the launch order and the batched
// launches (the device code is in hotpath_kernels.cuh; the odd-radix x
// lengths are instantiated in hotpath_odd.cu).
#include "hotpath_kernels.cuh"

namespace mm {

// Bit j set: pass (mode, stage) of tableau rk reads k_j (j >= 2).
unsigned stage_need_mask(int rk, int mode, int stage) {
    unsigned m = 0;
    if (rk < 0 || rk >= NRK) return 0;
    for (int j = 2; j <= 6 && j < stage; ++j) {
        bool need = false;
        if (mode == LM_RK) need = stage + 1 < 8 && h_rka[rk][stage + 1][j] != 0.0;
        else if (mode == LM_RKFINAL) need = h_rke[rk][j] != 0.0 || h_rkb[rk][j] != 0.0;
        if (need) m |= 1u << j;
    }
    return m;
}

__global__ void __launch_bounds__(256, 4) k_local(HotParams p, LaunchArgs a) {
    local_body<true>(p, a, blockIdx.x, gridDim.x);
}
// the cell pass of time steps (never evaluation mode: no energy sums)
__global__ void __launch_bounds__(256, 4) k_local_step(HotParams p, LaunchArgs a) {
    local_body<false>(p, a, blockIdx.x, gridDim.x);
}
// batched: work[b] = (sample, block of that sample, -, blocks of that sample)
__global__ void __launch_bounds__(256, 4)
kb_local(const HotParams* __restrict__ ps, const int4* __restrict__ work, LaunchArgs a) {
    const int4 w = work[blockIdx.x];
    __shared__ HotParams s_hp;
    load_params(ps + w.x, &s_hp);
    local_body<false>(s_hp, a, w.y, w.w);
}

// ---------------------------------------------------------------------------
__global__ void k_normalize_load(HotParams p, const float* __restrict__ m_user) {
    const long long n = p.ncell;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        st3(p.ms[0], i, n, normalized(ld3(m_user, i, n)));
}

// m_2 = m_n + h a21 k1 into mstage[0] (used when there is no x pass to fuse it into)
__global__ void k_combine2(HotParams p) {
    const DevState* st = p.st;
    if (st->done) return;
    const long long n = p.ncell;
    const int cur = st->cur;
    const Coef c = split(st->h * c_rka[p.rk][2][1]);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        st3(p.mstage[0], i, n, axpy(c, ld3(p.ks[cur], i, n), ld3(p.ms[cur], i, n)));
}

// Euler step of size st->h (set by the k1 pass): m_{n+1} = normalised(m_n + h k1),
// then one thread advances the clock and flips the state slots
__global__ void k_euler_update(HotParams p) {
    const DevState* st = p.st;
    if (st->done) return;
    const long long n = p.ncell;
    const int cur = st->cur;
    const Coef c = split(st->h);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        st3(p.ms[1 - cur], i, n, normalized(axpy(c, ld3(p.ks[cur], i, n), ld3(p.ms[cur], i, n))));
}

__global__ void k_euler_finish(HotParams p) {
    DevState* st = p.st;
    if (st->done) return;
    st->t += st->h;
    st->cur ^= 1;
    st->step_index += 1;
    st->accepted += 1;
    if (st->t_end > 0.0 && st->t >= st->t_end * (1.0 - 1e-12)) st->done = 1;
}

__global__ void k_copy_out(HotParams p, float* __restrict__ m_user) {
    const long long n = p.ncell;
    const float* src = p.ms[p.st->cur];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3 * n; i += (long long)gridDim.x * blockDim.x)
        m_user[i] = src[i];
}

// the 2-D column pass of 1024- and 2048-point lines runs the radix-16 register
// kernel (measured 38.7 against 43.7 us for the radix-8 one on the 2048-point
// column pass of the 1024^2 film); other lengths keep the radix-8 kernel
constexpr int CC16_MIN_LOGP = 10, CC16_MAX_LOGP = 11;

template <int L, int V>
static cudaError_t set_attr_batched_xy() {
    cudaError_t e;
    const int mx = 200 * 1024;
    if ((e = cudaFuncSetAttribute(kb_xfwd_r<L, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(kb_xinv_h<L, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(kb_colconv<L, 0, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(kb_yfwd<L, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    return cudaFuncSetAttribute(kb_yinv<L, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

template <int L>
static cudaError_t set_attr_all() {
    cudaError_t e;
    const int mx = 200 * 1024;
    if ((e = cudaFuncSetAttribute(k_xfwd<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_colconv<L, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_colconv<L, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if constexpr (L >= CC16_MIN_LOGP && L <= CC16_MAX_LOGP)
        if ((e = cudaFuncSetAttribute(k_colconv16<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_yfwd<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_yinv<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_xinv_local<L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_xinv_local<L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if constexpr (L >= LITE_MIN_LOGP) {
        if ((e = cudaFuncSetAttribute(k_xinv_local<L, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)))
            return e;
        if ((e = cudaFuncSetAttribute(k_xinv_local<L, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)))
            return e;
    }
    if constexpr (L >= XREG_MIN_LOGP && L <= XREG_MAX_LOGP) {
        if ((e = cudaFuncSetAttribute(k_xfwd_r<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
        if ((e = cudaFuncSetAttribute(k_xinv_h<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    }
    if constexpr (L >= BATCH_MIN_LOGP && L <= BATCH_MAX_LOGP) {
        if ((e = set_attr_batched_xy<L, 0>())) return e;
        if ((e = set_attr_batched_xy<L, 1>())) return e;
    }
    if constexpr (L >= 1 && L <= BATCH_MAX_LOGP) {
        if ((e = cudaFuncSetAttribute(kb_colconv<L, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
        if ((e = cudaFuncSetAttribute(kb_colconv<L, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    }
    if constexpr (L > 0) return set_attr_all<L - 1>();
    return cudaSuccess;
}

cudaError_t configure_hot_kernels() {
    cudaError_t e = set_attr_all<12>();
    if (e != cudaSuccess) return e;
    if ((e = configure_odd_kernels()) != cudaSuccess) return e;
    if ((e = configure_odd_yz_kernels()) != cudaSuccess) return e;
    if ((e = configure_yz_kernels()) != cudaSuccess) return e;
    return configure_small_kernels();
}

template <int L>
static void launch_x(const HotParams& p, const LaunchArgs& a, int pass, cudaStream_t s) {
    if constexpr (L >= XREG_MIN_LOGP && L <= XREG_MAX_LOGP) {
        using R = XR<L>;
        const dim3 g((p.ny + R::TY - 1) / R::TY, p.nz);
        // a time step in the fused layout transforms with the fused kernel's own
        // radix-16 passes, so that a spectrum is the same bits whichever pass made it
        const bool fused_step = a.mode != LM_EVAL && !p.hbuf;
        if (pass == PASS_XFWD && !fused_step) { k_xfwd_r<L><<<g, R::NT, R::SMEM, s>>>(p, a); return; }
        if (pass == PASS_XFWD_NEXT) {
            LaunchArgs b = a;
            b.src = a.next_src;
            k_xfwd_r<L><<<g, R::NT, R::SMEM, s>>>(p, b);
            return;
        }
        if (pass == PASS_XINV_H) { k_xinv_h<L><<<g, R::NT, R::SMEM, s>>>(p, a); return; }
    }
    using S = XS<L>;
    const dim3 g((p.ny + S::TY - 1) / S::TY, p.nz);
    const size_t sm = (size_t)S::NL * S::LS * sizeof(float2);
    if (pass == PASS_XFWD) { k_xfwd<L><<<g, S::NT, sm, s>>>(p, a); return; }
    if constexpr (L >= LITE_MIN_LOGP) {
        if (lite_terms(p)) {
            if (pass == PASS_XINV_LOCAL) k_xinv_local<L, false, true><<<g, S::NT, sm, s>>>(p, a);
            else k_xinv_local<L, true, true><<<g, S::NT, sm, s>>>(p, a);
            return;
        }
    }
    if (pass == PASS_XINV_LOCAL) k_xinv_local<L, false><<<g, S::NT, sm, s>>>(p, a);
    else k_xinv_local<L, true><<<g, S::NT, sm, s>>>(p, a);
}

template <int L>
static void launch_y(const HotParams& p, const LaunchArgs& a, int pass, cudaStream_t s) {
    if constexpr (L >= CC16_MIN_LOGP && L <= CC16_MAX_LOGP) {
        if (pass == PASS_YCONV) {
            using S = CC16<L>;
            k_colconv16<L><<<p.hx, S::NT, (size_t)3 * S::LS * sizeof(float2), s>>>(p, a);
            return;
        }
    }
    if (pass == PASS_YCONV) {
        using S = CC<L>;
        const dim3 g((p.hx + S::COLS - 1) / S::COLS);
        k_colconv<L, 0><<<g, S::NT, (size_t)3 * S::COLS * S::LS * sizeof(float2), s>>>(p, a);
    } else {
        using S = YS<L>;
        const dim3 g(p.hx, (p.nz + tz_of(L) - 1) / tz_of(L));
        const size_t sm = S::SMEM;
        if (pass == PASS_YFWD) k_yfwd<L><<<g, S::NT, sm, s>>>(p, a);
        else k_yinv<L><<<g, S::NT, sm, s>>>(p, a);
    }
}

template <int L>
static void launch_z(const HotParams& p, const LaunchArgs& a, cudaStream_t s) {
    using S = CC<L>;
    const dim3 g(p.hx, (p.py + S::COLS - 1) / S::COLS);
    k_colconv<L, 1><<<g, S::NT, (size_t)3 * S::COLS * S::LS * sizeof(float2), s>>>(p, a);
}

#define MM_LOGP_SWITCH(LOGP, CALL)                                          \
    switch (LOGP) {                                                         \
        case 0: CALL(0); break;   case 1: CALL(1); break;                   \
        case 2: CALL(2); break;   case 3: CALL(3); break;                   \
        case 4: CALL(4); break;   case 5: CALL(5); break;                   \
        case 6: CALL(6); break;   case 7: CALL(7); break;                   \
        case 8: CALL(8); break;   case 9: CALL(9); break;                   \
        case 10: CALL(10); break; case 11: CALL(11); break;                 \
        case 12: CALL(12); break;                                           \
        default: return cudaErrorInvalidValue;                              \
    }

#define MM_LOGP_SWITCH_INT(LOGP, CALL)                                      \
    switch (LOGP) {                                                         \
        case 0: CALL(0); break;   case 1: CALL(1); break;                   \
        case 2: CALL(2); break;   case 3: CALL(3); break;                   \
        case 4: CALL(4); break;   case 5: CALL(5); break;                   \
        case 6: CALL(6); break;   case 7: CALL(7); break;                   \
        case 8: CALL(8); break;   case 9: CALL(9); break;                   \
        case 10: CALL(10); break; case 11: CALL(11); break;                 \
        case 12: CALL(12); break;                                           \
        default: break;                                                     \
    }

int eval_passes(const HotParams& p, const LaunchArgs& a, int* ids) {
    int n = 0;
    if (p.demag && p.small_cl > 0) {
        ids[n++] = PASS_SMALL;          // every evaluation transforms its own input
        return n;
    }
    if (p.demag) {
        if (!a.have_spectrum) ids[n++] = PASS_XFWD;
        if (p.nz == 1) {
            ids[n++] = PASS_YCONV;
        } else if (yz_fused_nz(p)) {
            ids[n++] = PASS_YZCONV;
        } else {
            ids[n++] = PASS_YFWD;
            ids[n++] = PASS_ZCONV;
            ids[n++] = PASS_YINV;
        }
        if (p.rx == 1 && p.logpx >= XREG_MIN_LOGP && p.logpx <= XREG_MAX_LOGP && a.mode != LM_EVAL && p.hbuf) {
            // a step: inverse x transform, cell pass, forward x transform of the next input
            ids[n++] = PASS_XINV_H;
            ids[n++] = PASS_LOCAL_H;
            if (a.fuse) ids[n++] = PASS_XFWD_NEXT;
        } else {
            ids[n++] = a.fuse ? PASS_XINV_FUSED : PASS_XINV_LOCAL;
        }
    } else {
        if (a.src == SRC_COMBINE2) ids[n++] = PASS_COMBINE2;   // no x pass to fold m_2 into
        ids[n++] = PASS_LOCAL;
    }
    return n;
}

cudaError_t launch_pass(const HotParams& p, const LaunchArgs& a, int pass, cudaStream_t s) {
    switch (pass) {
        case PASS_XFWD:
        case PASS_XINV_LOCAL:
        case PASS_XINV_FUSED:
        case PASS_XINV_H:
        case PASS_XFWD_NEXT:
            if (p.rx > 1) return launch_x_mixed(p, a, pass, s);
#define MM_CALL_X(L) launch_x<L>(p, a, pass, s)
            MM_LOGP_SWITCH(p.logpx, MM_CALL_X)
#undef MM_CALL_X
            break;
        case PASS_YCONV:
        case PASS_YFWD:
        case PASS_YINV:
            if (p.ry > 1) return launch_yz_mixed(p, a, pass, s);
#define MM_CALL_Y(L) launch_y<L>(p, a, pass, s)
            MM_LOGP_SWITCH(p.logpy, MM_CALL_Y)
#undef MM_CALL_Y
            break;
        case PASS_ZCONV:
            if (p.zsplit) return launch_zconv_split(p, a, s);
            if (p.rz > 1) return launch_yz_mixed(p, a, pass, s);
#define MM_CALL_Z(L) launch_z<L>(p, a, s)
            MM_LOGP_SWITCH(p.logpz, MM_CALL_Z)
#undef MM_CALL_Z
            break;
        case PASS_COMBINE2:
            k_combine2<<<4 * 152, 256, 0, s>>>(p);
            break;
        case PASS_SMALL:
            return launch_small(p, a, s);
        case PASS_YZCONV:
            return launch_yzconv(p, a, s);
        case PASS_LOCAL:            // one cell per thread: every load in flight at once
            k_local<<<(unsigned)((p.ncell + 255) / 256), 256, 0, s>>>(p, a);
            break;
        case PASS_LOCAL_H:          // time steps only
            k_local_step<<<(unsigned)((p.ncell + 255) / 256), 256, 0, s>>>(p, a);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched passes.  One launch covers the blocks of many independent samples
// that share the pass's FFT length; work[b] = (sample, block x, block y,
// blocks of that sample in this pass).  The block bodies are the ones of the
// single-sample kernels, so a sample's result does not depend on the batch.

int batch_pass_logp(const HotParams& p, int pass) {
    switch (pass) {
        case PASS_XFWD: case PASS_XFWD_NEXT: case PASS_XINV_H: return p.logpx;
        case PASS_YCONV: case PASS_YFWD: case PASS_YINV: return p.logpy;
        case PASS_ZCONV: return p.logpz;
        case PASS_YZCONV: return p.logpy * 100 + yz_fused_nz(p);     // length and z cells per block
        default: return 0;
    }
}

bool batch_supported(const HotParams& p) {
    if (!p.demag) return false;
    if (p.rx != 1 || p.ry != 1 || p.rz != 1) return false;      // odd-radix lengths: single contexts only
    if (p.logpx < BATCH_MIN_LOGP || p.logpx > BATCH_MAX_LOGP) return false;
    if (p.logpy < BATCH_MIN_LOGP || p.logpy > BATCH_MAX_LOGP) return false;
    if (p.nz > 1 && (p.logpz < 1 || p.logpz > BATCH_MAX_LOGP)) return false;
    return true;
}

cudaError_t batch_pass_grid(const HotParams& p, int pass, int variant, int* gx, int* gy) {
    *gx = 0;
    *gy = 0;
    switch (pass) {
        case PASS_XFWD: case PASS_XFWD_NEXT: case PASS_XINV_H:
            if (variant == 2) {
#define MM_G(L) { *gx = (p.ny + XR<L, 1>::TY - 1) / XR<L, 1>::TY; *gy = p.nz; }
                MM_LOGP_SWITCH(p.logpx, MM_G)
#undef MM_G
                return cudaSuccess;
            }
#define MM_G(L) { *gx = (p.ny + XR<L>::TY - 1) / XR<L>::TY; *gy = p.nz; }
            MM_LOGP_SWITCH(p.logpx, MM_G)
#undef MM_G
            return cudaSuccess;
        case PASS_YCONV:
            if (p.nz != 1) return cudaSuccess;
#define MM_G(L) { *gx = (p.hx + CC<L>::COLS - 1) / CC<L>::COLS; *gy = 1; }
            MM_LOGP_SWITCH(p.logpy, MM_G)
#undef MM_G
            return cudaSuccess;
        case PASS_YZCONV:
            if (p.nz == 1 || !yz_fused_nz(p)) return cudaSuccess;
            *gx = p.hx;
            *gy = 1;
            return cudaSuccess;
        case PASS_YFWD: case PASS_YINV:
            if (p.nz == 1 || yz_fused_nz(p)) return cudaSuccess;
            *gx = p.hx;
            *gy = (p.nz + tz_of(p.logpy) - 1) / tz_of(p.logpy);
            return cudaSuccess;
        case PASS_ZCONV:
            if (p.nz == 1 || yz_fused_nz(p)) return cudaSuccess;
#define MM_G(L) { *gx = p.hx; *gy = (p.py + CC<L>::COLS - 1) / CC<L>::COLS; }
            MM_LOGP_SWITCH(p.logpz, MM_G)
#undef MM_G
            return cudaSuccess;
        case PASS_LOCAL_H:
            *gx = (int)((p.ncell + 255) / 256);
            *gy = 1;
            return cudaSuccess;
        default:
            return cudaErrorInvalidValue;
    }
}

template <int L, int V>
static cudaError_t launch_b(const HotParams* ps, const int4* work, int nb, const LaunchArgs& a, int pass,
                            cudaStream_t s) {
    if constexpr (V == 2) {
        // the half tile exists for the register x passes only
        if constexpr (L >= BATCH_MIN_LOGP && L <= BATCH_MAX_LOGP) {
            using R = XR<L, 1>;
            switch (pass) {
                case PASS_XFWD:
                    kb_xfwd_r<L, 2><<<nb, R::NT, R::SMEM, s>>>(ps, work, a);
                    return cudaSuccess;
                case PASS_XFWD_NEXT: {
                    LaunchArgs b = a;
                    b.src = a.next_src;
                    kb_xfwd_r<L, 2><<<nb, R::NT, R::SMEM, s>>>(ps, work, b);
                    return cudaSuccess;
                }
                case PASS_XINV_H:
                    kb_xinv_h<L, 2><<<nb, R::NT, R::SMEM, s>>>(ps, work, a);
                    return cudaSuccess;
                default: break;
            }
        }
        return cudaErrorInvalidValue;
    }
    if constexpr (L >= BATCH_MIN_LOGP && L <= BATCH_MAX_LOGP) {
        switch (pass) {
            case PASS_XFWD:
                kb_xfwd_r<L, V><<<nb, XR<L>::NT, XR<L>::SMEM, s>>>(ps, work, a);
                return cudaSuccess;
            case PASS_XFWD_NEXT: {
                LaunchArgs b = a;
                b.src = a.next_src;
                kb_xfwd_r<L, V><<<nb, XR<L>::NT, XR<L>::SMEM, s>>>(ps, work, b);
                return cudaSuccess;
            }
            case PASS_XINV_H:
                kb_xinv_h<L, V><<<nb, XR<L>::NT, XR<L>::SMEM, s>>>(ps, work, a);
                return cudaSuccess;
            case PASS_YCONV:
                kb_colconv<L, 0, V><<<nb, CC<L>::NT, (size_t)3 * CC<L>::COLS * CC<L>::LS * sizeof(float2), s>>>(ps, work, a);
                return cudaSuccess;
            case PASS_YFWD: case PASS_YINV: {
                using S = YS<L>;
                const size_t sm = S::SMEM;
                if (pass == PASS_YFWD) kb_yfwd<L, V><<<nb, S::NT, sm, s>>>(ps, work, a);
                else kb_yinv<L, V><<<nb, S::NT, sm, s>>>(ps, work, a);
                return cudaSuccess;
            }
            default: break;
        }
    }
    if constexpr (L >= 1 && L <= BATCH_MAX_LOGP) {
        if (pass == PASS_ZCONV) {
            kb_colconv<L, 1, V><<<nb, CC<L>::NT, (size_t)3 * CC<L>::COLS * CC<L>::LS * sizeof(float2), s>>>(ps, work, a);
            return cudaSuccess;
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_pass_batched(const HotParams* ps, const int4* work, int nb, const LaunchArgs& a, int pass,
                                int logp, int variant, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (pass == PASS_LOCAL_H) {
        kb_local<<<nb, 256, 0, s>>>(ps, work, a);
        return cudaGetLastError();
    }
    if (pass == PASS_YZCONV) return launch_yzconv_batched(ps, work, nb, a, logp, s);
    if (variant == 2) {
#define MM_CALL_B(L) e = launch_b<L, 2>(ps, work, nb, a, pass, s)
        MM_LOGP_SWITCH(logp, MM_CALL_B)
#undef MM_CALL_B
    } else if (variant) {
#define MM_CALL_B(L) e = launch_b<L, 1>(ps, work, nb, a, pass, s)
        MM_LOGP_SWITCH(logp, MM_CALL_B)
#undef MM_CALL_B
    } else {
#define MM_CALL_B(L) e = launch_b<L, 0>(ps, work, nb, a, pass, s)
        MM_LOGP_SWITCH(logp, MM_CALL_B)
#undef MM_CALL_B
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// number of compiled register budgets of a batched pass at this FFT length
// (1 where both budgets give the same kernel)
int batch_variants(int pass, int logp) {
    int n = 1;
    switch (pass) {
        case PASS_XFWD: case PASS_XFWD_NEXT: case PASS_XINV_H:
            // variants 0 and 1: register budgets; 2: half the row pairs per block
#define MM_V(L) n = XR<L, 1>::PAIRS < XR<L>::PAIRS ? 3 : (XR<L>::MINB1 != XR<L>::MINB ? 2 : 1)
            MM_LOGP_SWITCH_INT(logp, MM_V)
#undef MM_V
            break;
        case PASS_YCONV: case PASS_ZCONV:
#define MM_V(L) n = CC<L>::MINB1 != CC<L>::MINB0 ? 2 : 1
            MM_LOGP_SWITCH_INT(logp, MM_V)
#undef MM_V
            break;
        case PASS_YFWD: case PASS_YINV:
#define MM_V(L) n = YS<L>::MINB1 != YS<L>::MINB ? 2 : 1
            MM_LOGP_SWITCH_INT(logp, MM_V)
#undef MM_V
            break;
        default: break;
    }
    return n;
}

// copies every sample's DevState into one array (one thread per sample)
__global__ void k_gather_states(const HotParams* __restrict__ ps, DevState* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = *ps[i].st;
}

__global__ void k_set_run_batch(const HotParams* __restrict__ ps, const int* __restrict__ active, int n,
                                double tol, double torque_tol, double dt0_s, int fixed_h) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const HotParams& p = ps[active[k]];
    DevState* st = p.st;
    st->tol = tol;
    st->fixed_h = fixed_h;
    st->t_end = 0.0;
    st->torque_tol = torque_tol;
    st->max_dm = 0.0;
    st->h_cap = 0.0;
    if (dt0_s > 0.0) st->h = dt0_s * p.t_unit;
    st->h_min = 1e-20 * p.t_unit;
    st->done = 0;
    st->status = 0;
}

cudaError_t launch_set_run_batch(const HotParams* ps, const int* active, int n_active, double tol,
                                 double torque_tol, double dt0_s, int fixed_h, cudaStream_t s) {
    if (n_active <= 0) return cudaSuccess;
    k_set_run_batch<<<(n_active + 127) / 128, 128, 0, s>>>(ps, active, n_active, tol, torque_tol, dt0_s, fixed_h);
    return cudaGetLastError();
}

cudaError_t launch_gather_states(const HotParams* ps, DevState* out, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_gather_states<<<(n + 127) / 128, 128, 0, s>>>(ps, out, n);
    return cudaGetLastError();
}

cudaError_t launch_normalize_load(const HotParams& p, const float* m_user, cudaStream_t s) {
    k_normalize_load<<<4 * 152, 256, 0, s>>>(p, m_user);
    return cudaGetLastError();
}

cudaError_t launch_euler_update(const HotParams& p, cudaStream_t s) {
    const long long blocks = (p.ncell + 255) / 256;
    k_euler_update<<<(unsigned)(blocks < 4 * 152 ? blocks : 4 * 152), 256, 0, s>>>(p);
    k_euler_finish<<<1, 1, 0, s>>>(p);
    return cudaGetLastError();
}

// m_user -> state slot 0 as it is (no renormalisation: a checkpoint resumes bit for bit)
__global__ void k_copy_in(HotParams p, const float* __restrict__ m_user) {
    const long long n = 3 * p.ncell;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p.ms[0][i] = m_user[i];
}

cudaError_t launch_copy_in(const HotParams& p, const float* m_user, cudaStream_t s) {
    k_copy_in<<<4 * 152, 256, 0, s>>>(p, m_user);
    return cudaGetLastError();
}

cudaError_t launch_copy_out(const HotParams& p, float* m_user, cudaStream_t s) {
    k_copy_out<<<4 * 152, 256, 0, s>>>(p, m_user);
    return cudaGetLastError();
}

}  // namespace mm
