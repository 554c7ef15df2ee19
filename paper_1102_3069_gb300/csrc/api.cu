// api.cu - the C ABI of include/mm.h: context, workspace layout, argument
// checks and the order of kernel launches for an evaluation or a step.
#include "mm.h"
#include "mm_internal.cuh"
#include "fft32.cuh"

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <string>
#include <vector>

namespace {

constexpr double MU0 = 4.0e-7 * M_PI;
constexpr double KB = 1.380649e-23;
constexpr double DEFAULT_GAMMA0 = 2.211e5;

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Runge-Kutta methods of the C ABI -> tableau index, stages, first-same-as-last, adaptive
struct RkInfo { int index, stages, fsal, adaptive; };
bool rk_info(int method, RkInfo* r) {
    switch (method) {
        case MM_RKDP: *r = {0, 7, 1, 1}; return true;
        case MM_RK23: *r = {1, 4, 1, 1}; return true;
        case MM_RKCK: *r = {2, 6, 0, 1}; return true;
        case MM_RK4:  *r = {3, 4, 0, 0}; return true;
        case MM_RK3:  *r = {4, 3, 0, 0}; return true;
        case MM_RK12: *r = {5, 2, 0, 1}; return true;
        default: return false;
    }
}
bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }
int next_pow2(int v) { int p = 1; while (p < v) p <<= 1; return p; }
// compiled passes for the length r * 2^l along axis a
bool odd_supported(int axis, int r, int l) {
    return axis == 0 ? mm::odd_x_length_supported(r, l) : mm::odd_yz_length_supported(r, l);
}
// v = r * 2^l with r = 3, 5 or 7 and compiled passes for that length along axis a
bool odd_length(int v, int axis, int* r_out) {
    int l = 0;
    while (v > 1 && (v & 1) == 0) { v >>= 1; ++l; }
    if (v != 3 && v != 5 && v != 7) return false;
    if (!odd_supported(axis, v, l)) return false;
    *r_out = v;
    return true;
}
// FFT length of an axis of n cells: periodic - n itself (2^k or r 2^l);
// open - the smallest 2^k, or with odd factors allowed r 2^l, >= 2n - 1
bool pad_length(int n, bool periodic, int axis, bool odd, int* P, int* R) {
    *R = 1;
    if (periodic) {
        *P = n;
        return (is_pow2(n) && n <= 4096) || odd_length(n, axis, R);
    }
    if (n > 2048) return false;
    *P = next_pow2(2 * n - 1);
    if (odd)
        for (int r = 3; r <= 7; r += 2)
            for (int l = 0; (r << l) <= 4096; ++l)
                if ((r << l) >= 2 * n - 1 && (r << l) < *P && odd_supported(axis, r, l)) {
                    *P = r << l;
                    *R = r;
                }
    return true;
}

// Gauss-Legendre nodes/weights on [-1, 1] (Newton iteration on P_n)
void gauss_legendre(int n, double* t, double* w) {
    for (int i = 0; i < n; ++i) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        t[i] = x;
        w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

}  // namespace

struct mm_ctx {
    // geometry
    int nx = 0, ny = 0, nz = 0;
    double dx = 0, dy = 0, dz = 0;
    int pbc[3] = {0, 0, 0};
    int images = 0;
    int px = 1, py = 1, pz = 1, logpx = 0, logpy = 0, logpz = 0;
    int rx = 1, ry = 1, rz = 1;     // odd factor of each padded length (r * 2^logp)
    size_t off_twr[8] = {0};        // exp(-2 pi i t / (r TWN)) tables of the odd factors in use
    int hx = 1, hyk = 1, hzk = 1, nyp = 16, nzp = 1, ty = 2, tz = 1, tky = 1, kxb = 1, ncomp = 4;
    int ox = 1, oy = 1, oz = 1;
    long long ncell = 0;
    cudaStream_t stream = nullptr;
    // material
    bool have_material = false;
    double Ms = 0, Aex = 0, Ku = 0, u[3] = {1, 0, 0}, alpha = 0, gamma0 = DEFAULT_GAMMA0, T = 0;
    uint64_t seed = 0;
    double B[3] = {0, 0, 0};
    double K1 = 0, K2 = 0, cub[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    double stt_P = 0, stt_xi = 0, stt_j[3] = {0, 0, 0};
    const float* uaxis = nullptr;   // per-cell easy axes (caller-owned device array) or null
    bool demag = true;
    bool kernel_ready = false;
    // workspace
    char* ws = nullptr;
    size_t ws_size = 0;
    size_t off_st = 0, off_tw = 0, off_kt = 0, off_s1 = 0, off_s2 = 0, off_union = 0;
    size_t sz_kt = 0, sz_s1 = 0, sz_s2 = 0, sz_rk = 0, sz_setup = 0, total = 0;
    // integrator bookkeeping
    bool state_loaded = false;
    bool k1_valid = false;
    bool rk_h_set = false;          // an RKDP step size has been given since mm_load
    int last_method = 0;
    bool last_maxdm = false;        // the last run chose its steps by the maximum variation of m
    double max_dm = 0.0;            // mm_set_max_dm (0: fixed dt)
    int layout = MM_LAYOUT_AUTO;    // mm_set_pass_layout
    int dft_prec = MM_DFT_FP32;     // mm_set_dft_precision
    size_t off_zs = 0, sz_zs = 0, zs_sizes[7] = {0, 0, 0, 0, 0, 0, 0};
    // what the x spectrum in the workspace currently holds: nothing usable, the
    // transform of m_n (ms[cur]) or of the Dormand-Prince stage-2 input m_2
    enum { SPEC_NONE, SPEC_MCUR, SPEC_M2 } spec = SPEC_NONE;
    double last_fixed_dt = 0.0;     // internal units
    long long step_counter = 0;
    uint64_t th_step = 0;
    double th_dt = 0.0;            // seconds
    std::vector<float2> tw_host;
    std::string err;
    // one standard step captured as a CUDA graph and replayed (see mm_advance)
    cudaGraphExec_t step_graph = nullptr;
    // while set, eval() records its launch arguments here instead of launching
    std::vector<mm::LaunchArgs>* rec = nullptr;
    int graph_method = 0;
    double graph_dt = 0.0;
    unsigned long long graph_version = 0;
    unsigned long long param_version = 1;   // bumped whenever launch parameters change
    // per-pass event timing (mm_profile / mm_pass_times)
    struct Rec { int pass; cudaEvent_t a, b; };
    bool profiling = false;
    std::vector<Rec> prof;
    double pass_ms[mm::NPASS] = {0};
    long long pass_n[mm::NPASS] = {0};
};

namespace {

int fail(mm_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(mm_ctx* c, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, MM_ECUDA, m);
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
    } while (0)

void layout(mm_ctx* c) {
    const long long n3 = 3 * c->ncell;
    c->sz_kt = (size_t)c->ncomp * c->hx * c->hyk * c->hzk * sizeof(float);
    c->sz_s1 = (size_t)3 * c->hx * c->nz * c->nyp * sizeof(float2);
    c->sz_s2 = c->nz > 1 ? (size_t)3 * c->hx * c->py * c->nzp * sizeof(float2) : 0;
    // ms[2], ks[2], k2..k6, mstage[2], hbuf: 12 arrays of 3*ncell floats
    c->sz_rk = 12 * align256((size_t)n3 * sizeof(float));
    c->sz_setup = align256((size_t)6 * c->ox * c->oy * c->oz * sizeof(double)) +
                  align256((size_t)c->px * c->py * c->pz * sizeof(double2));
    size_t off = 0;
    c->off_st = off; off += align256(sizeof(mm::DevState));
    c->off_tw = off; off += align256((size_t)mmfft::TWN * sizeof(float2));
    for (int r = 3; r <= 7; r += 2) {
        c->off_twr[r] = 0;
        if (c->rx == r || c->ry == r || c->rz == r) {
            c->off_twr[r] = off;
            off += align256((size_t)r * mmfft::TWN * sizeof(float2));
        }
    }
    c->off_kt = off; off += align256(c->sz_kt);
    c->off_s1 = off; off += align256(c->sz_s1);
    c->off_s2 = off; off += align256(c->sz_s2);
    c->off_union = off; off += (c->sz_rk > c->sz_setup ? c->sz_rk : c->sz_setup);
    c->sz_zs = c->dft_prec == MM_DFT_SPLIT_BF16
                   ? mm::zsplit_bytes(c->nx, c->ny, c->nz, c->hx, c->py, c->pz, c->nzp, c->zs_sizes)
                   : 0;
    c->off_zs = off; off += align256(c->sz_zs);
    c->total = off;
}

// FFT lengths r * 2^logp of the three axes and what follows from them
void set_lengths(mm_ctx* c, const int P[3], const int R[3]) {
    c->px = P[0]; c->py = P[1]; c->pz = P[2];
    c->rx = R[0]; c->ry = R[1]; c->rz = R[2];
    c->logpx = ilog2(P[0] / R[0]); c->logpy = ilog2(P[1] / R[1]); c->logpz = ilog2(P[2] / R[2]);
    c->hx = c->px / 2 + 1;
    if (c->px == 1) c->hx = 1;
    c->hyk = c->py / 2 + 1;
    c->hzk = c->pz / 2 + 1;
    // launch shapes: the kernels' compile-time tiles (fft32.cuh)
    c->ty = mmfft::ty_of(c->logpx);
    c->tz = c->ry > 1 ? mmfft::tz_of_len(c->py) : mmfft::tz_of(c->logpy);
    c->nzp = (c->nz + c->tz - 1) / c->tz * c->tz;  // the 3-D y passes write whole z tiles
}

mm::DevState* dstate(mm_ctx* c) { return reinterpret_cast<mm::DevState*>(c->ws + c->off_st); }

float* rk_array(mm_ctx* c, int i) {
    const size_t each = align256((size_t)3 * c->ncell * sizeof(float));
    return reinterpret_cast<float*>(c->ws + c->off_union + i * each);
}

int check_ready(mm_ctx* ctx, bool need_kernel) {
    if (!ctx) return MM_EINVAL;
    if (!ctx->ws) return fail(ctx, MM_ENOMEM, "workspace not set (mm_set_workspace)");
    if (!ctx->have_material) return fail(ctx, MM_ESTATE, "material not set (mm_set_material)");
    if (need_kernel && ctx->demag && !ctx->kernel_ready)
        return fail(ctx, MM_ESTATE, "demag kernel not built (mm_demag_kernel) or demag not disabled");
    return MM_OK;
}

// Whether MM_LAYOUT_AUTO takes the one-launch cluster evaluation for a grid
// that fits it (cl > 0 CTAs).  Not for now: on GB300 it measured slower than
// the multi-kernel passes at every size it applies to (32^2 Euler 29.8 against
// 22.6 us per step, 128^2 36.2 against 30.8 us, 256^2 113 against 32 us):
// each CTA runs the phases of an evaluation one after another, and the chain
// of barriers and dependent latencies is longer than the multi-kernel passes'
// launch gaps.
bool small_auto(const mm::HotParams& p, int cl) {
    (void)p;
    (void)cl;
    return false;
}

mm::HotParams hot_params(mm_ctx* c, double dt_internal, bool thermal) {
    mm::HotParams p;
    std::memset(&p, 0, sizeof(p));
    p.nx = c->nx; p.ny = c->ny; p.nz = c->nz;
    p.px = c->px; p.py = c->py; p.pz = c->pz;
    p.logpx = c->logpx; p.logpy = c->logpy; p.logpz = c->logpz;
    p.hx = c->hx; p.hyk = c->hyk; p.hzk = c->hzk;
    p.nyp = c->nyp; p.nzp = c->nzp;
    p.ty = c->ty; p.tz = c->tz; p.tky = c->tky; p.kxb = c->kxb;
    for (int i = 0; i < 3; ++i) p.pbc[i] = c->pbc[i];
    p.ncomp = c->ncomp;
    p.ncell = c->ncell;
    const double Ms = c->Ms;
    const double ex = 2.0 * c->Aex / (MU0 * Ms * Ms);
    p.cex[0] = (float)(ex / (c->dx * c->dx));
    p.cex[1] = (float)(ex / (c->dy * c->dy));
    p.cex[2] = (float)(ex / (c->dz * c->dz));
    p.kan = (float)(2.0 * c->Ku / (MU0 * Ms * Ms));
    p.ux = (float)c->u[0]; p.uy = (float)c->u[1]; p.uz = (float)c->u[2];
    p.uaxis = c->uaxis;
    p.hzx = (float)(c->B[0] / (MU0 * Ms));
    p.hzy = (float)(c->B[1] / (MU0 * Ms));
    p.hzz = (float)(c->B[2] / (MU0 * Ms));
    p.kc1 = (float)(2.0 * c->K1 / (MU0 * Ms * Ms));
    p.kc2 = (float)(2.0 * c->K2 / (MU0 * Ms * Ms));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) p.c[i][j] = (float)c->cub[i][j];
    if (c->stt_P != 0.0 && (c->stt_j[0] != 0.0 || c->stt_j[1] != 0.0 || c->stt_j[2] != 0.0)) {
        constexpr double MU_B = 9.2740100783e-24, E_CHARGE = 1.602176634e-19;
        const double bj = c->stt_P * MU_B / (E_CHARGE * Ms * (1.0 + c->stt_xi * c->stt_xi));
        const double d[3] = {c->dx, c->dy, c->dz};
        for (int a = 0; a < 3; ++a) p.stt_s[a] = (float)(bj * c->stt_j[a] / (2.0 * d[a] * c->gamma0 * Ms));
        p.stt_beta = (float)(c->stt_xi - c->alpha);
        p.stt = 1;
    }
    p.alpha = (float)c->alpha;
    p.llpref = (float)(1.0 / (1.0 + c->alpha * c->alpha));
    p.seed = c->seed;
    p.demag = c->demag ? 1 : 0;
    p.dt_d = dt_internal;
    if (thermal && c->T > 0.0 && dt_internal > 0.0) {
        const double dt_s = dt_internal / (c->gamma0 * Ms);
        const double V = c->dx * c->dy * c->dz;
        const double sigma = std::sqrt(2.0 * c->alpha * KB * c->T / (c->gamma0 * MU0 * Ms * V * dt_s));
        p.sigma_th = (float)(sigma / Ms);
    }
    p.h_scale = (float)Ms;
    p.t_scale = (float)(c->gamma0 * Ms);
    p.t_unit = c->gamma0 * Ms;
    p.tw = reinterpret_cast<const float2*>(c->ws + c->off_tw);
    p.rx = c->rx; p.ry = c->ry; p.rz = c->rz;
    for (int r = 3; r <= 7; r += 2)
        if (c->off_twr[r]) p.twr[r] = reinterpret_cast<const float2*>(c->ws + c->off_twr[r]);
    p.kt = reinterpret_cast<const float*>(c->ws + c->off_kt);
    p.s1 = reinterpret_cast<float2*>(c->ws + c->off_s1);
    p.s2 = reinterpret_cast<float2*>(c->ws + c->off_s2);
    p.st = dstate(c);
    p.ms[0] = rk_array(c, 0); p.ms[1] = rk_array(c, 1);
    p.ks[0] = rk_array(c, 2); p.ks[1] = rk_array(c, 3);
    for (int j = 2; j <= 6; ++j) p.kb[j] = rk_array(c, 2 + j);    // 4..8
    p.mstage[0] = rk_array(c, 9); p.mstage[1] = rk_array(c, 10);
    p.hbuf = rk_array(c, 11);
    if (c->dft_prec == MM_DFT_SPLIT_BF16) {
        // [A hi | A lo | X | Y hi | Y lo | O | F hi | F lo | G hi | G lo | error word]
        const size_t* z = c->zs_sizes;
        char* b = c->ws + c->off_zs;
        p.zsplit = 1;
        p.zs_kp = 2 * c->nzp;
        p.zs_a_hi = b; b += z[0];
        p.zs_a_lo = b; b += z[0];
        p.zs_x = reinterpret_cast<float*>(b); b += z[1];
        p.zs_y_hi = b; b += z[2];
        p.zs_y_lo = b; b += z[2];
        p.zs_o = reinterpret_cast<float*>(b); b += z[3];
        p.zs_f_hi = b; b += z[4];
        p.zs_f_lo = b; b += z[4];
        p.zs_g_hi = b; b += z[4];
        p.zs_g_lo = b; b += z[4];
        p.zs_err = reinterpret_cast<unsigned*>(b);
    }
    // small 2-D grids: one cluster launch per evaluation (automatic, or forced)
    if (c->demag && (c->layout == MM_LAYOUT_AUTO || c->layout == MM_LAYOUT_CLUSTER)) {
        const int cl = mm::small_cluster_size(p);
        if (c->layout == MM_LAYOUT_CLUSTER || small_auto(p, cl)) p.small_cl = cl;
    }
    return p;
}

// run parameters are written by a one-thread kernel so that mm_advance stays asynchronous
__global__ void k_set_run(mm::DevState* st, double tol, double t_end, double torque_tol, double h,
                          double h_min, int reset_done, int fixed_h, double max_dm, double h_cap) {
    st->tol = tol;
    st->max_dm = max_dm;
    st->h_cap = h_cap;
    st->fixed_h = fixed_h;
    st->t_end = t_end;
    st->torque_tol = torque_tol;
    if (h > 0.0) st->h = h;
    st->h_min = h_min;
    if (reset_done) { st->done = 0; st->status = 0; }
    if (st->t_end > 0.0 && st->h > st->t_end - st->t) st->h = st->t_end - st->t;
}

mm::LaunchArgs make_args(const mm::HotParams& p, int src, int mode, int stage, bool fuse, bool have_spectrum) {
    mm::LaunchArgs a{src, mode, stage, fuse ? 1 : 0, have_spectrum ? 1 : 0};
    // where the cell pass leaves the next evaluation's input (what a fused
    // forward x transform reads): after Euler and Heun's second stage the
    // last block has already flipped the slots, so m_{n+1} is ms[cur]
    switch (mode) {
        case mm::LM_K1: case mm::LM_HEUN1: a.next_src = mm::SRC_STAGE0; break;
        case mm::LM_RK:
            a.next_src = (p.rk_fsal && stage + 1 == p.rk_stages) ? mm::SRC_NEXT
                       : (((stage + 1) & 1) ? mm::SRC_STAGE1 : mm::SRC_STAGE0);
            break;
        case mm::LM_EULER: case mm::LM_HEUN2: a.next_src = mm::SRC_CUR; a.keep = 1; break;
        default: a.next_src = mm::SRC_CUR; break;
    }
    a.need = mm::stage_need_mask(p.rk, mode, stage);
    return a;
}

// Which x-pass layout a time step uses (where the FFT length allows both):
// split (inverse x, cell pass, forward x of the next input: three launches,
// H_demag through HBM) or fused (one kernel).  The automatic choice is the
// fused kernel: measured faster for every method (1024^2 film, Dormand-Prince
// 0.736 against 0.773 ms per step, Euler 0.127 against 0.136 ms; 256x256x64
// cube, Heun 0.632 against 0.668 ms).  Batches always run the split passes.
bool use_split_layout(const mm_ctx* ctx, int method, bool maxdm) {
    (void)method;
    (void)maxdm;
    return ctx->layout == MM_LAYOUT_SPLIT;
}

int eval(mm_ctx* ctx, const mm::HotParams& p, int src, int mode, int stage, bool fuse = false,
         bool have_spectrum = false) {
    const mm::LaunchArgs a = make_args(p, src, mode, stage, fuse, have_spectrum);
    if (ctx->rec) {
        ctx->rec->push_back(a);
        return MM_OK;
    }
    int ids[8];
    const int n = mm::eval_passes(p, a, ids);
    for (int i = 0; i < n; ++i) {
        if (!ctx->profiling) {
            CK(mm::launch_pass(p, a, ids[i], ctx->stream));
            continue;
        }
        // the context owns the pair as soon as both exist: mm_pass_times and
        // mm_destroy release them on every path
        mm_ctx::Rec r{ids[i], nullptr, nullptr};
        cudaError_t e = cudaEventCreate(&r.a);
        if (e == cudaSuccess) e = cudaEventCreate(&r.b);
        if (e != cudaSuccess) {
            if (r.a) cudaEventDestroy(r.a);
            return cuda_fail(ctx, e, "cudaEventCreate");
        }
        ctx->prof.push_back(r);
        CK(cudaEventRecord(r.a, ctx->stream));
        CK(mm::launch_pass(p, a, ids[i], ctx->stream));
        CK(cudaEventRecord(r.b, ctx->stream));
    }
    return MM_OK;
}

}  // namespace

namespace {

// The launches of one time step.  The standard step (first = false) finds
// no usable spectrum for RKDP stage 2 (the new h is only known on the device)
// and finds the spectrum of m_n in place for Euler/Heun (the previous step's
// fused pass made it).  The first step of a run is the other way round:
// right after k1 the stage-2 input and its spectrum are in place (RKDP), and
// right after a load nothing is (Euler/Heun).
int enqueue_step(mm_ctx* ctx, const mm::HotParams& p, int method, bool first) {
    int rc;
    RkInfo r;
    if (ctx->max_dm > 0.0 && (method == MM_EULER || method == MM_HEUN || (rk_info(method, &r) && !r.adaptive))) {
        // fixed maximum variation of m per step: the k1 pass reduces max |k1|
        // and its last block sets h; the stage-2 input is then formed by the
        // forward x pass (m_n + h a21 k1) with that h
        if ((rc = eval(ctx, p, mm::SRC_CUR, mm::LM_K1, 1, false, false))) return rc;
        if (method == MM_EULER) {
            CK(mm::launch_euler_update(p, ctx->stream));
            return MM_OK;
        }
        const int S = p.rk_stages;
        auto src_of = [&](int st) { return (st & 1) ? mm::SRC_STAGE1 : mm::SRC_STAGE0; };
        if (S == 2) return eval(ctx, p, mm::SRC_COMBINE2, mm::LM_RKFINAL, 2, false, false);
        if ((rc = eval(ctx, p, mm::SRC_COMBINE2, mm::LM_RK, 2, true, false))) return rc;
        for (int st = 3; st < S; ++st)
            if ((rc = eval(ctx, p, src_of(st), mm::LM_RK, st, true, true))) return rc;
        return eval(ctx, p, src_of(S), mm::LM_RKFINAL, S, false, true);
    }
    if (rk_info(method, &r)) {
        const int S = r.stages;
        // stage s reads its input from mstage[s & 1]; with first same as last
        // the last stage reads the candidate m_{n+1} (slot ms[1-cur])
        auto src_of = [&](int st) { return (st & 1) ? mm::SRC_STAGE1 : mm::SRC_STAGE0; };
        if (r.fsal) {
            if ((rc = eval(ctx, p, mm::SRC_COMBINE2, mm::LM_RK, 2, true, first))) return rc;
            for (int st = 3; st < S; ++st)
                if ((rc = eval(ctx, p, src_of(st), mm::LM_RK, st, true, true))) return rc;
            return eval(ctx, p, mm::SRC_NEXT, mm::LM_RKFINAL, S, false, true);
        }
        // without first same as last: k1 = f(m_n) each step (the pass also forms m_2)
        if ((rc = eval(ctx, p, mm::SRC_CUR, mm::LM_K1, 1, true, first))) return rc;
        for (int st = 2; st < S; ++st)
            if ((rc = eval(ctx, p, src_of(st), mm::LM_RK, st, true, true))) return rc;
        return eval(ctx, p, src_of(S), mm::LM_RKFINAL, S, false, true);
    }
    if (method == MM_EULER) return eval(ctx, p, mm::SRC_CUR, mm::LM_EULER, 0, true, !first);
    if ((rc = eval(ctx, p, mm::SRC_CUR, mm::LM_HEUN1, 0, true, !first))) return rc;
    return eval(ctx, p, mm::SRC_STAGE0, mm::LM_HEUN2, 0, true, true);
}

}  // namespace

// ---------------------------------------------------------------------------
// Scratch for mm_eval_heff_static: one fixed array per GPU, reserved when the
// library's module is loaded on that device and held until the process exits.
// Layout: [DevState | twiddle table | x spectrum | y spectrum (3-D only)].
static __device__ __align__(256) unsigned char g_static_scratch[MM_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
void* g_static_ptr[kMaxDevices] = {nullptr};

// Once per device, with that device current: look up the device address of
// the scratch array (in host code its name is only a host-side stand-in) and
// fill the constant twiddle table it carries.
int static_scratch_for_current_device(mm_ctx* ctx, char** out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(ctx, MM_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[dev]) {
        void* ptr = nullptr;
        CK(cudaGetSymbolAddress(&ptr, g_static_scratch));
        CK(mm::configure_hot_kernels());
        CK(cudaMemcpy(static_cast<char*>(ptr) + align256(sizeof(mm::DevState)), ctx->tw_host.data(),
                      mmfft::TWN * sizeof(float2), cudaMemcpyHostToDevice));
        g_static_ptr[dev] = ptr;
    }
    *out = static_cast<char*>(g_static_ptr[dev]);
    return MM_OK;
}

}  // namespace

extern "C" {

int mm_init_geometry(mm_ctx** out, int nx, int ny, int nz, double dx, double dy, double dz, int pbc_x, int pbc_y,
                     int pbc_z, int pbc_images, void* cuda_stream) {
    if (!out) return MM_EINVAL;
    *out = nullptr;
    const int n[3] = {nx, ny, nz};
    const int pb[3] = {pbc_x != 0, pbc_y != 0, pbc_z != 0};
    int P[3], R[3];
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1) return MM_EINVAL;
        if (!pad_length(n[a], pb[a], a, true, &P[a], &R[a])) return MM_EINVAL;
    }
    if (!(dx > 0 && dy > 0 && dz > 0) || !std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(dz))
        return MM_EINVAL;
    if (pbc_images < 0 || pbc_images > 1000) return MM_EINVAL;
    mm_ctx* c = new (std::nothrow) mm_ctx();
    if (!c) return MM_ENOMEM;
    c->nx = nx; c->ny = ny; c->nz = nz;
    c->dx = dx; c->dy = dy; c->dz = dz;
    for (int a = 0; a < 3; ++a) c->pbc[a] = pb[a];
    c->images = pbc_images;
    set_lengths(c, P, R);
    c->ncomp = nz == 1 ? 4 : 6;
    c->ncell = (long long)nx * ny * nz;
    c->ox = pb[0] ? nx / 2 + 1 : nx;
    c->oy = pb[1] ? ny / 2 + 1 : ny;
    c->oz = pb[2] ? nz / 2 + 1 : nz;
    // launch shapes: the kernels' compile-time tiles (fft32.cuh), about 384
    // threads per block with one radix-16 butterfly each
    c->nyp = (ny + 15) / 16 * 16;                  // a multiple of every x-pass tile
    c->kxb = 1;                                    // column passes size their own blocks
    c->tky = 1;
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    layout(c);
    // twiddle table, rounded once from double
    c->tw_host.resize(mmfft::TWN);
    for (int t = 0; t < mmfft::TWN; ++t) {
        const double a = -2.0 * M_PI * (double)t / (double)mmfft::TWN;
        c->tw_host[t] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    *out = c;
    return MM_OK;
}

size_t mm_workspace_bytes(const mm_ctx* ctx) { return ctx ? ctx->total : 0; }

size_t mm_demag_tensor_len(const mm_ctx* ctx) { return ctx ? (size_t)6 * ctx->ox * ctx->oy * ctx->oz : 0; }

int mm_set_workspace(mm_ctx* ctx, void* dev_ptr, size_t bytes) {
    if (!ctx || !dev_ptr) return fail(ctx, MM_EINVAL, "null workspace");
    if (reinterpret_cast<uintptr_t>(dev_ptr) & 255) return fail(ctx, MM_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < ctx->total) return fail(ctx, MM_ENOMEM, "workspace smaller than mm_workspace_bytes()");
    // opt every hot kernel into large dynamic shared memory (once per process and device)
    {
        static std::atomic<unsigned long long> configured_mask{0};
        int dev = 0;
        CK(cudaGetDevice(&dev));
        const unsigned long long bit = (dev >= 0 && dev < 64) ? 1ull << dev : 0ull;   // 0: configure every time
        if (!(configured_mask.load() & bit)) {
            CK(mm::configure_hot_kernels());
            configured_mask.fetch_or(bit);
        }
    }
    ctx->ws = static_cast<char*>(dev_ptr);
    ctx->ws_size = bytes;
    CK(cudaMemcpyAsync(ctx->ws + ctx->off_tw, ctx->tw_host.data(), mmfft::TWN * sizeof(float2),
                       cudaMemcpyHostToDevice, ctx->stream));
    std::vector<float2> twr;
    for (int r = 3; r <= 7; r += 2) {
        if (!ctx->off_twr[r]) continue;
        twr.resize((size_t)r * mmfft::TWN);
        for (int t = 0; t < r * mmfft::TWN; ++t) {
            const double a = -2.0 * M_PI * (double)t / ((double)r * mmfft::TWN);
            twr[t] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
        CK(cudaMemcpyAsync(ctx->ws + ctx->off_twr[r], twr.data(), twr.size() * sizeof(float2),
                           cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));      // twr is reused for the next table
    }
    CK(cudaMemsetAsync(ctx->ws + ctx->off_st, 0, sizeof(mm::DevState), ctx->stream));
    if (ctx->dft_prec == MM_DFT_SPLIT_BF16) {
        CK(cudaMemsetAsync(ctx->ws + ctx->off_zs, 0, ctx->sz_zs, ctx->stream));
        CK(mm::zsplit_tables(hot_params(ctx, 0.0, false), ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->kernel_ready = false;
    ctx->state_loaded = false;
    ctx->spec = mm_ctx::SPEC_NONE;
    ctx->param_version++;
    return MM_OK;
}

int mm_set_material(mm_ctx* ctx, double Ms, double Aex, double Ku, const double easy_axis[3], double alpha,
                    double gamma0, double temperature, uint64_t seed, const double B_applied_T[3]) {
    if (!ctx) return MM_EINVAL;
    if (!(Ms > 0) || !std::isfinite(Ms)) return fail(ctx, MM_EINVAL, "Ms must be > 0");
    if (!(Aex >= 0) || !std::isfinite(Aex)) return fail(ctx, MM_EINVAL, "Aex must be >= 0");
    if (!std::isfinite(Ku)) return fail(ctx, MM_EINVAL, "Ku must be finite");
    if (!(alpha >= 0) || !std::isfinite(alpha)) return fail(ctx, MM_EINVAL, "alpha must be >= 0");
    if (gamma0 == 0.0) gamma0 = DEFAULT_GAMMA0;
    if (!(gamma0 > 0) || !std::isfinite(gamma0)) return fail(ctx, MM_EINVAL, "gamma0 must be > 0");
    if (!(temperature >= 0) || !std::isfinite(temperature)) return fail(ctx, MM_EINVAL, "temperature must be >= 0");
    double u[3] = {1, 0, 0};
    if (Ku != 0.0) {
        if (!easy_axis) return fail(ctx, MM_EINVAL, "easy axis needed when Ku != 0");
        const double n = std::sqrt(easy_axis[0] * easy_axis[0] + easy_axis[1] * easy_axis[1] + easy_axis[2] * easy_axis[2]);
        if (!(n > 0) || !std::isfinite(n)) return fail(ctx, MM_EINVAL, "easy axis must be a non-zero vector");
        for (int i = 0; i < 3; ++i) u[i] = easy_axis[i] / n;
    }
    double B[3] = {0, 0, 0};
    if (B_applied_T)
        for (int i = 0; i < 3; ++i) {
            if (!std::isfinite(B_applied_T[i])) return fail(ctx, MM_EINVAL, "applied field must be finite");
            B[i] = B_applied_T[i];
        }
    const bool ms_changed = ctx->have_material && ctx->Ms != Ms;
    ctx->Ms = Ms; ctx->Aex = Aex; ctx->Ku = Ku; ctx->alpha = alpha; ctx->gamma0 = gamma0; ctx->T = temperature;
    ctx->seed = seed;
    for (int i = 0; i < 3; ++i) { ctx->u[i] = u[i]; ctx->B[i] = B[i]; }
    ctx->have_material = true;
    if (ms_changed) ctx->state_loaded = false;     // internal time unit changed
    ctx->k1_valid = false;
    ctx->param_version++;
    return MM_OK;
}

int mm_set_cubic_anisotropy(mm_ctx* ctx, double K1, double K2, const double c1[3], const double c2[3]) {
    if (!ctx) return MM_EINVAL;
    if (!std::isfinite(K1) || !std::isfinite(K2)) return fail(ctx, MM_EINVAL, "K1, K2 must be finite");
    double a[3] = {1, 0, 0}, b[3] = {0, 1, 0};
    if (K1 != 0.0 || K2 != 0.0) {
        if (!c1 || !c2) return fail(ctx, MM_EINVAL, "cubic axes needed when K1 or K2 != 0");
        for (int i = 0; i < 3; ++i) { a[i] = c1[i]; b[i] = c2[i]; }
    }
    // Gram-Schmidt: c1 normalised, c2 made orthogonal to it, c3 = c1 x c2
    const double na = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    if (!(na > 0) || !std::isfinite(na)) return fail(ctx, MM_EINVAL, "cubic axis c1 must be a non-zero vector");
    for (int i = 0; i < 3; ++i) a[i] /= na;
    const double d = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    for (int i = 0; i < 3; ++i) b[i] -= d * a[i];
    const double nb = std::sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    if (!(nb > 1e-12 * (1.0 + std::fabs(d))) || !std::isfinite(nb))
        return fail(ctx, MM_EINVAL, "cubic axis c2 must not be parallel to c1");
    for (int i = 0; i < 3; ++i) b[i] /= nb;
    const double c3[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    for (int i = 0; i < 3; ++i) { ctx->cub[0][i] = a[i]; ctx->cub[1][i] = b[i]; ctx->cub[2][i] = c3[i]; }
    ctx->K1 = K1;
    ctx->K2 = K2;
    ctx->k1_valid = false;
    ctx->param_version++;
    return MM_OK;
}

int mm_set_stt(mm_ctx* ctx, double P, double xi, const double j_A_per_m2[3]) {
    if (!ctx) return MM_EINVAL;
    if (!std::isfinite(P) || !std::isfinite(xi)) return fail(ctx, MM_EINVAL, "P and xi must be finite");
    double j[3] = {0, 0, 0};
    if (j_A_per_m2)
        for (int a = 0; a < 3; ++a) {
            if (!std::isfinite(j_A_per_m2[a])) return fail(ctx, MM_EINVAL, "current density must be finite");
            j[a] = j_A_per_m2[a];
        }
    ctx->stt_P = P;
    ctx->stt_xi = xi;
    for (int a = 0; a < 3; ++a) ctx->stt_j[a] = j[a];
    ctx->k1_valid = false;
    ctx->param_version++;
    return MM_OK;
}

int mm_set_anisotropy_axes(mm_ctx* ctx, const float* u) {
    if (!ctx) return MM_EINVAL;
    if (u && (reinterpret_cast<uintptr_t>(u) & 3)) return fail(ctx, MM_EINVAL, "axis array must be float aligned");
    ctx->uaxis = u;
    ctx->k1_valid = false;
    ctx->param_version++;
    return MM_OK;
}

int mm_set_fft_lengths(mm_ctx* ctx, int mode) {
    if (!ctx) return MM_EINVAL;
    if (mode != MM_FFT_2357 && mode != MM_FFT_POW2) return fail(ctx, MM_EINVAL, "mode must be MM_FFT_2357 or MM_FFT_POW2");
    if (ctx->ws) return fail(ctx, MM_ESTATE, "the FFT lengths are chosen before mm_set_workspace");
    const int n[3] = {ctx->nx, ctx->ny, ctx->nz};
    int P[3], R[3];
    for (int a = 0; a < 3; ++a)
        if (!pad_length(n[a], ctx->pbc[a] != 0, a, mode == MM_FFT_2357, &P[a], &R[a]))
            return fail(ctx, MM_EINVAL, "no FFT length for this axis");
    if (mode == MM_FFT_POW2 && (R[0] > 1 || R[1] > 1 || R[2] > 1))
        return fail(ctx, MM_EINVAL, "a periodic axis of r * 2^l cells needs its odd factor");
    set_lengths(ctx, P, R);
    layout(ctx);
    return MM_OK;
}

int mm_set_dft_precision(mm_ctx* ctx, int mode) {
    if (!ctx) return MM_EINVAL;
    if (mode != MM_DFT_FP32 && mode != MM_DFT_SPLIT_BF16)
        return fail(ctx, MM_EINVAL, "mode must be MM_DFT_FP32 or MM_DFT_SPLIT_BF16");
    if (ctx->ws) return fail(ctx, MM_ESTATE, "the DFT precision is chosen before mm_set_workspace");
    if (mode == MM_DFT_SPLIT_BF16 && (ctx->nz < 2 || ctx->pz < 4))
        return fail(ctx, MM_EINVAL, "the split-BF16 z pass needs a 3-D grid with a padded z length >= 4");
    ctx->dft_prec = mode;
    layout(ctx);
    return MM_OK;
}

int mm_set_pass_layout(mm_ctx* ctx, int layout) {
    if (!ctx) return MM_EINVAL;
    if (layout != MM_LAYOUT_AUTO && layout != MM_LAYOUT_FUSED && layout != MM_LAYOUT_SPLIT &&
        layout != MM_LAYOUT_CLUSTER)
        return fail(ctx, MM_EINVAL,
                    "layout must be MM_LAYOUT_AUTO, MM_LAYOUT_FUSED, MM_LAYOUT_SPLIT or MM_LAYOUT_CLUSTER");
    if (layout == MM_LAYOUT_CLUSTER) {
        mm::HotParams q;
        std::memset(&q, 0, sizeof(q));
        q.nx = ctx->nx; q.ny = ctx->ny; q.nz = ctx->nz;
        q.logpx = ctx->logpx; q.logpy = ctx->logpy;
        q.rx = ctx->rx; q.ry = ctx->ry;
        for (int i = 0; i < 3; ++i) q.pbc[i] = ctx->pbc[i];
        q.ncell = ctx->ncell;
        if (mm::small_cluster_size(q) == 0)
            return fail(ctx, MM_EINVAL, "MM_LAYOUT_CLUSTER needs a 2-D grid (open z) with power-of-two FFT lengths "
                                        "whose half spectrum fits 16 CTAs' shared memory");
    }
    if (layout != ctx->layout) {
        ctx->layout = layout;
        ctx->k1_valid = false;
        ctx->spec = mm_ctx::SPEC_NONE;
        ctx->param_version++;
    }
    return MM_OK;
}

int mm_set_max_dm(mm_ctx* ctx, double max_dm) {
    if (!ctx) return MM_EINVAL;
    if (!(max_dm >= 0.0) || !std::isfinite(max_dm) || max_dm > 1.0)
        return fail(ctx, MM_EINVAL, "max_dm must be in [0, 1]");
    ctx->max_dm = max_dm;
    ctx->k1_valid = false;
    ctx->param_version++;
    return MM_OK;
}

int mm_set_demag(mm_ctx* ctx, int enabled) {
    if (!ctx) return MM_EINVAL;
    ctx->demag = enabled != 0;
    ctx->k1_valid = false;
    ctx->param_version++;
    return MM_OK;
}

int mm_demag_kernel(mm_ctx* ctx, double* out_tensor_host) {
    if (!ctx) return MM_EINVAL;
    if (!ctx->ws) return fail(ctx, MM_ENOMEM, "workspace not set (mm_set_workspace)");
    mm::SetupParams p;
    std::memset(&p, 0, sizeof(p));
    p.nx = ctx->nx; p.ny = ctx->ny; p.nz = ctx->nz;
    p.px = ctx->px; p.py = ctx->py; p.pz = ctx->pz;
    p.ox = ctx->ox; p.oy = ctx->oy; p.oz = ctx->oz;
    for (int i = 0; i < 3; ++i) p.pbc[i] = ctx->pbc[i];
    p.images = ctx->images;
    p.ncomp = ctx->ncomp;
    p.hx = ctx->hx; p.hyk = ctx->hyk; p.hzk = ctx->hzk;
    const double dmax = std::fmax(ctx->dx, std::fmax(ctx->dy, ctx->dz));
    p.dx = ctx->dx / dmax; p.dy = ctx->dy / dmax; p.dz = ctx->dz / dmax;
    const int orders[4] = {3, 4, 6, 8};
    for (int q = 0; q < 4; ++q) {
        p.gl_n[q] = orders[q];
        gauss_legendre(orders[q], p.gl_t[q], p.gl_w[q]);
    }
    const size_t oct_bytes = (size_t)6 * ctx->ox * ctx->oy * ctx->oz * sizeof(double);
    p.oct = reinterpret_cast<double*>(ctx->ws + ctx->off_union);
    p.work = reinterpret_cast<double2*>(ctx->ws + ctx->off_union + align256(oct_bytes));
    p.kt = reinterpret_cast<float*>(ctx->ws + ctx->off_kt);
    p.st = dstate(ctx);
    ctx->state_loaded = false;
    ctx->k1_valid = false;
    ctx->spec = mm_ctx::SPEC_NONE;
    ctx->param_version++;
    CK(cudaMemsetAsync(&p.st->kre_bits, 0, 2 * sizeof(unsigned long long), ctx->stream));
    CK(mm::launch_kernel_setup(p, ctx->stream));
    if (out_tensor_host) CK(cudaMemcpyAsync(out_tensor_host, p.oct, oct_bytes, cudaMemcpyDeviceToHost, ctx->stream));
    unsigned long long bits[2];
    CK(cudaMemcpyAsync(bits, &p.st->kre_bits, sizeof(bits), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double re, im;
    std::memcpy(&re, &bits[0], 8);
    std::memcpy(&im, &bits[1], 8);
    if (!(re > 0) || !std::isfinite(re) || !std::isfinite(im))
        return fail(ctx, MM_ENONFINITE, "demag kernel setup produced non-finite values");
    if (im > 1e-9 * re) {
        char buf[128];
        std::snprintf(buf, sizeof(buf), "demag kernel spectrum not real: |Im|/|Re| = %.3g", im / re);
        return fail(ctx, MM_ENONFINITE, buf);
    }
    ctx->kernel_ready = true;
    return MM_OK;
}

int mm_set_thermal_clock(mm_ctx* ctx, uint64_t step_index, double dt_s) {
    if (!ctx) return MM_EINVAL;
    if (!(dt_s >= 0) || !std::isfinite(dt_s)) return fail(ctx, MM_EINVAL, "dt must be >= 0");
    ctx->th_step = step_index;
    ctx->th_dt = dt_s;
    return MM_OK;
}

int mm_eval_heff(mm_ctx* ctx, const float* m, float* h_out, float* torque_out, double* energy_J_host) {
    int rc = check_ready(ctx, true);
    if (rc) return rc;
    if (!m) return fail(ctx, MM_EINVAL, "null m");
    const double tu = ctx->gamma0 * ctx->Ms;
    mm::HotParams p = hot_params(ctx, ctx->th_dt * tu, true);
    p.m_eval = m;
    p.h_out = h_out;
    p.tq_out = torque_out;
    p.want_energy = energy_J_host != nullptr;
    p.thermal_step = (long long)ctx->th_step;
    mm::DevState* st = dstate(ctx);
    CK(cudaMemsetAsync(&st->energy_acc, 0, sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(&st->tsq_acc, 0, sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(&st->status, 0, sizeof(int), ctx->stream));
    ctx->spec = mm_ctx::SPEC_NONE;          // the evaluation reuses the spectrum buffer
    rc = eval(ctx, p, mm::SRC_PTR, mm::LM_EVAL, 0);
    if (rc) return rc;
    if (energy_J_host) {
        double acc = 0.0;
        int status = 0;
        CK(cudaMemcpyAsync(&acc, &st->energy_acc, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(&status, &st->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        const double V = ctx->dx * ctx->dy * ctx->dz;
        *energy_J_host = MU0 * ctx->Ms * ctx->Ms * V * acc;
        if (status == MM_ENONFINITE) return fail(ctx, MM_ENONFINITE, "non-finite effective field");
    }
    return MM_OK;
}

int mm_load(mm_ctx* ctx, const float* m, double t0_s, uint64_t step_index) {
    int rc = check_ready(ctx, false);
    if (rc) return rc;
    if (!m) return fail(ctx, MM_EINVAL, "null m");
    if (!std::isfinite(t0_s)) return fail(ctx, MM_EINVAL, "t0 must be finite");
    mm::DevState h;
    std::memset(&h, 0, sizeof(h));
    h.t = t0_s * ctx->gamma0 * ctx->Ms;
    h.step_index = (long long)step_index;
    mm::DevState* st = dstate(ctx);
    CK(cudaMemcpyAsync(st, &h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
    mm::HotParams p = hot_params(ctx, 0.0, false);
    CK(mm::launch_normalize_load(p, m, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));       // h lives on this stack frame
    ctx->state_loaded = true;
    ctx->k1_valid = false;
    ctx->rk_h_set = false;
    ctx->spec = mm_ctx::SPEC_NONE;
    ctx->step_counter = (long long)step_index;
    return MM_OK;
}

int mm_store(mm_ctx* ctx, float* m) {
    if (!ctx) return MM_EINVAL;
    if (!ctx->state_loaded) return fail(ctx, MM_ESTATE, "no state loaded (mm_load)");
    if (!m) return fail(ctx, MM_EINVAL, "null m");
    mm::HotParams p = hot_params(ctx, 0.0, false);
    CK(mm::launch_copy_out(p, m, ctx->stream));
    return MM_OK;
}

int mm_advance(mm_ctx* ctx, int method, long nsteps, double dt_s, double tol, double t_end_s, double torque_tol) {
    int rc = check_ready(ctx, true);
    if (rc) return rc;
    if (!ctx->state_loaded) return fail(ctx, MM_ESTATE, "no state loaded (mm_load)");
    if (nsteps < 0) return fail(ctx, MM_EINVAL, "nsteps must be >= 0");
    if (!std::isfinite(dt_s) || !std::isfinite(tol) || !std::isfinite(t_end_s) || !std::isfinite(torque_tol))
        return fail(ctx, MM_EINVAL, "non-finite argument");
    const double tu = ctx->gamma0 * ctx->Ms;
    RkInfo rk = {0, 7, 1, 1};
    bool is_rk = rk_info(method, &rk);
    // the methods without an error estimate take a fixed dt or, with
    // mm_set_max_dm, the step that moves the fastest cell by max_dm
    const bool maxdm = ctx->max_dm > 0.0 && (method == MM_EULER || method == MM_HEUN || (is_rk && !rk.adaptive));
    if (maxdm) {
        if (ctx->T > 0.0) return fail(ctx, MM_EINVAL, "thermal field needs a fixed dt (maximum-variation steps vary it)");
        if (!(dt_s >= 0)) return fail(ctx, MM_EINVAL, "dt (the step cap) must be >= 0");
        if (method == MM_HEUN) { rk = {6, 2, 0, 0}; is_rk = true; }     // Heun as a two-stage tableau
        if (method == MM_EULER) rk = {6, 2, 0, 0};                     // only its k1 pass runs
    } else if (method == MM_EULER || method == MM_HEUN || (is_rk && !rk.adaptive)) {
        if (!(dt_s > 0)) return fail(ctx, MM_EINVAL, "fixed-step methods need dt > 0");
    } else if (is_rk) {
        if (ctx->T > 0.0) return fail(ctx, MM_EINVAL, "thermal field needs a fixed-step method (fixed dt)");
        if (tol == 0.0) return fail(ctx, MM_EINVAL, "adaptive methods need tol > 0 (or < 0 for fixed steps)");
        if (tol < 0.0 && !(dt_s > 0)) return fail(ctx, MM_EINVAL, "fixed steps (tol < 0) need dt > 0");
    } else {
        return fail(ctx, MM_EINVAL, "unknown method");
    }
    double dt = dt_s * tu;
    if (is_rk && rk.adaptive) {
        if (dt > 0) ctx->rk_h_set = true;
        else if (!ctx->rk_h_set) { dt = 1e-13 * tu; ctx->rk_h_set = true; }   // default first step 100 fs
    }
    ctx->last_method = method;
    mm::HotParams p = hot_params(ctx, dt, true);
    p.rk = rk.index;
    p.rk_stages = rk.stages;
    p.rk_fsal = rk.fsal;
    if (!use_split_layout(ctx, method, maxdm)) p.hbuf = nullptr;   // the fused x passes
    const bool fixed_steps = (is_rk && (!rk.adaptive || tol < 0.0)) || maxdm;
    k_set_run<<<1, 1, 0, ctx->stream>>>(dstate(ctx), fixed_steps ? 1.0 : tol, t_end_s > 0 ? t_end_s * tu : 0.0,
                                        torque_tol > 0 ? torque_tol : 0.0,
                                        (is_rk || maxdm) ? (dt > 0 ? dt : 0.0) : 0.0, 1e-20 * tu, 1,
                                        fixed_steps ? 1 : 0, maxdm ? ctx->max_dm : 0.0,
                                        maxdm && dt > 0 ? dt : 0.0);
    CK(cudaGetLastError());
    if (is_rk && rk.fsal) {
        if (dt > 0 && ctx->spec == mm_ctx::SPEC_M2) ctx->spec = mm_ctx::SPEC_NONE;   // m_2 depends on h
        if (!ctx->k1_valid) {
            // k1 = f(m_n); the same pass forms m_2 and its x spectrum
            if ((rc = eval(ctx, p, mm::SRC_CUR, mm::LM_K1, 1, true, ctx->spec == mm_ctx::SPEC_MCUR))) return rc;
            ctx->k1_valid = true;
            ctx->spec = mm_ctx::SPEC_M2;
        }
    } else {
        ctx->k1_valid = false;
        ctx->last_fixed_dt = dt;
    }
    long s = 0;
    // a first step that can reuse a spectrum already in place differs from
    // the standard step: launch it directly
    // FSAL tableaus: right after k1 the stage-2 input and its spectrum are in place;
    // others: the first step finds the spectrum of m_n in place only if a previous
    // Euler/Heun run left it (their standard step needs it, the tableaus' does not)
    ctx->last_maxdm = maxdm;
    bool first_special;
    if (maxdm) first_special = false;              // every step starts from its own k1 pass
    else if (is_rk && rk.fsal) first_special = ctx->spec == mm_ctx::SPEC_M2;
    else if (is_rk) first_special = ctx->spec == mm_ctx::SPEC_MCUR;
    else first_special = ctx->spec != mm_ctx::SPEC_MCUR;
    if (nsteps > 0 && first_special) {
        if ((rc = enqueue_step(ctx, p, method, true))) return rc;
        ++s;
    }
    if (s < nsteps && p.small_cl > 0 && !maxdm && !ctx->profiling) {
        // small 2-D grids: every remaining standard step in one persistent cluster launch
        std::vector<mm::LaunchArgs> rec;
        ctx->rec = &rec;
        const int erc = enqueue_step(ctx, p, method, false);
        ctx->rec = nullptr;
        if (erc) return erc;
        if (!rec.empty() && rec.size() <= 8) {
            mm::SmallSteps L;
            std::memset(&L, 0, sizeof(L));
            L.nsteps = nsteps - s;
            L.n = (int)rec.size();
            for (int i = 0; i < L.n; ++i) L.a[i] = rec[i];
            CK(mm::launch_small_steps(p, L, ctx->stream));
            s = nsteps;
        }
    }
    if (s < nsteps) {
        // the standard step: replayed from a CUDA graph on a capturable stream
        bool graphed = false;
        if (ctx->stream != nullptr && !ctx->profiling) {
            if (!ctx->step_graph || ctx->graph_method != method || ctx->graph_version != ctx->param_version ||
                ctx->graph_dt != dt) {
                if (ctx->step_graph) { cudaGraphExecDestroy(ctx->step_graph); ctx->step_graph = nullptr; }
                cudaGraph_t g = nullptr;
                if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                    const int erc = enqueue_step(ctx, p, method, false);
                    const cudaError_t ee = cudaStreamEndCapture(ctx->stream, &g);
                    if (erc == MM_OK && ee == cudaSuccess && g &&
                        cudaGraphInstantiate(&ctx->step_graph, g, 0) == cudaSuccess) {
                        ctx->graph_method = method;
                        ctx->graph_dt = dt;
                        ctx->graph_version = ctx->param_version;
                    } else {
                        ctx->step_graph = nullptr;
                    }
                    if (g) cudaGraphDestroy(g);
                }
                cudaGetLastError();     // a refused capture leaves no sticky error
            }
            graphed = ctx->step_graph != nullptr;
        }
        for (; s < nsteps; ++s) {
            if (graphed) {
                CK(cudaGraphLaunch(ctx->step_graph, ctx->stream));
            } else if ((rc = enqueue_step(ctx, p, method, false))) {
                return rc;
            }
        }
    }
    // Euler/Heun leave the spectrum of the state slot in place, unless a torque
    // stop kept m_n after its pass had transformed the rejected new state
    if (nsteps > 0) ctx->spec = (is_rk || maxdm || torque_tol > 0.0) ? mm_ctx::SPEC_NONE : mm_ctx::SPEC_MCUR;
    if (is_rk && !rk.fsal) ctx->k1_valid = false;
    return MM_OK;
}

int mm_get_stats(mm_ctx* ctx, mm_stats* stats) {
    if (!ctx) return MM_EINVAL;
    if (!ctx->ws) return fail(ctx, MM_ENOMEM, "workspace not set");
    mm::DevState h;
    CK(cudaMemcpyAsync(&h, dstate(ctx), sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const double tu = ctx->gamma0 * ctx->Ms;
    ctx->step_counter = h.step_index;
    if (stats) {
        stats->evals = h.evals;
        stats->accepted = h.accepted;
        stats->rejected = h.rejected;
        stats->step_index = h.step_index;
        stats->t = h.t / tu;
        RkInfo ri;
        stats->dt = ((rk_info(ctx->last_method, &ri) && ri.adaptive) || ctx->last_maxdm ? h.h : ctx->last_fixed_dt) / tu;
        stats->last_err = h.last_err;
        stats->max_torque = h.max_torque;
        const double V = ctx->dx * ctx->dy * ctx->dz;
        stats->energy = MU0 * ctx->Ms * ctx->Ms * V * h.energy_acc;
        stats->dissipation = -MU0 * ctx->Ms * ctx->Ms * ctx->Ms * V * ctx->gamma0 * ctx->alpha /
                             (1.0 + ctx->alpha * ctx->alpha) * h.tsq_acc;
        stats->status = h.status;
        stats->done = h.done;
    }
    return MM_OK;
}

int mm_get_state(mm_ctx* ctx, float* m, mm_checkpoint* out) {
    if (!ctx) return MM_EINVAL;
    if (!ctx->state_loaded) return fail(ctx, MM_ESTATE, "no state loaded (mm_load)");
    if (!out) return fail(ctx, MM_EINVAL, "null checkpoint");
    if (m) {
        mm::HotParams p = hot_params(ctx, 0.0, false);
        CK(mm::launch_copy_out(p, m, ctx->stream));
    }
    mm::DevState h;
    CK(cudaMemcpyAsync(&h, dstate(ctx), sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const double tu = ctx->gamma0 * ctx->Ms;
    std::memset(out, 0, sizeof(*out));
    out->t = h.t / tu;
    out->dt = h.h / tu;
    out->step_index = h.step_index;
    out->accepted = h.accepted;
    out->rejected = h.rejected;
    out->evals = h.evals;
    out->after_reject = h.after_reject;
    out->t_internal = h.t;
    out->dt_internal = h.h;
    return MM_OK;
}

int mm_set_state(mm_ctx* ctx, const float* m, const mm_checkpoint* in) {
    int rc = check_ready(ctx, false);
    if (rc) return rc;
    if (!m || !in) return fail(ctx, MM_EINVAL, "null argument");
    if (!std::isfinite(in->t) || !std::isfinite(in->dt) || in->dt < 0.0 || in->step_index < 0 || in->accepted < 0 ||
        in->rejected < 0 || in->evals < 0)
        return fail(ctx, MM_EINVAL, "bad checkpoint");
    const double tu = ctx->gamma0 * ctx->Ms;
    mm::DevState h;
    std::memset(&h, 0, sizeof(h));
    h.t = in->t * tu;
    h.h = in->dt * tu;
    // the exact internal values when they are this checkpoint's (same time unit)
    if (std::isfinite(in->t_internal) && std::fabs(in->t_internal / tu - in->t) <= 1e-12 * std::fabs(in->t) + 1e-300)
        h.t = in->t_internal;
    if (std::isfinite(in->dt_internal) && in->dt_internal >= 0.0 &&
        std::fabs(in->dt_internal / tu - in->dt) <= 1e-12 * in->dt + 1e-300)
        h.h = in->dt_internal;
    h.step_index = in->step_index;
    h.accepted = in->accepted;
    h.rejected = in->rejected;
    h.evals = in->evals;
    h.after_reject = in->after_reject ? 1 : 0;
    mm::DevState* st = dstate(ctx);
    CK(cudaMemcpyAsync(st, &h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
    mm::HotParams p = hot_params(ctx, 0.0, false);
    CK(mm::launch_copy_in(p, m, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));       // h lives on this stack frame
    ctx->state_loaded = true;
    ctx->k1_valid = false;
    ctx->rk_h_set = in->dt > 0.0;
    ctx->spec = mm_ctx::SPEC_NONE;
    ctx->step_counter = in->step_index;
    return MM_OK;
}

int mm_step(mm_ctx* ctx, float* m, int method, double* t_s, double* dt_s, double tol, int* accepted) {
    if (!ctx) return MM_EINVAL;
    if (!m || !t_s || !dt_s) return fail(ctx, MM_EINVAL, "null argument");
    int rc = mm_load(ctx, m, *t_s, (uint64_t)ctx->step_counter);
    if (rc) return rc;
    if ((rc = mm_advance(ctx, method, 1, *dt_s, tol, 0.0, 0.0))) return rc;
    if ((rc = mm_store(ctx, m))) return rc;
    mm_stats s;
    if ((rc = mm_get_stats(ctx, &s))) return rc;
    if (s.status) return fail(ctx, s.status, s.status == MM_ENONFINITE ? "non-finite values in the step"
                                                                        : "step size underflow");
    if (accepted) *accepted = s.accepted > 0;
    *t_s = s.t;
    *dt_s = s.dt;
    return MM_OK;
}

int mm_relax(mm_ctx* ctx, float* m, double torque_tol, double err_tol, long max_steps, long* steps_out,
             double* torque_out) {
    if (!ctx) return MM_EINVAL;
    if (!m) return fail(ctx, MM_EINVAL, "null m");
    if (!(torque_tol > 0) || !(err_tol > 0) || max_steps < 0) return fail(ctx, MM_EINVAL, "bad relax arguments");
    int rc = mm_load(ctx, m, 0.0, 0);
    if (rc) return rc;
    mm_stats s;
    std::memset(&s, 0, sizeof(s));
    long done_steps = 0;
    bool first = true;
    while (true) {
        const long chunk = (max_steps - done_steps) < 64 ? (max_steps - done_steps) : 64;
        if ((rc = mm_advance(ctx, MM_RKDP, chunk, first ? 1e-13 : 0.0, err_tol, 0.0, torque_tol))) return rc;
        first = false;
        done_steps += chunk;
        if ((rc = mm_get_stats(ctx, &s))) return rc;
        if (s.done || done_steps >= max_steps) break;
    }
    if ((rc = mm_store(ctx, m))) return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    if (steps_out) *steps_out = (long)(s.accepted + s.rejected);
    if (torque_out) *torque_out = s.max_torque;
    if (s.status) return fail(ctx, s.status, "relaxation failed on the device");
    if (!(s.done && s.max_torque < torque_tol)) return fail(ctx, MM_ENOTCONVERGED, "torque bound not reached");
    return MM_OK;
}

int mm_run_host(mm_ctx* ctx, float* m_host, int method, long nsteps, double dt_s, double tol) {
    int rc = check_ready(ctx, true);
    if (rc) return rc;
    if (!m_host) return fail(ctx, MM_EINVAL, "null m");
    const size_t bytes = (size_t)3 * ctx->ncell * sizeof(float);
    // the second stage buffer doubles as the device copy of the caller's array
    float* dev = rk_array(ctx, 10);
    CK(cudaMemcpyAsync(dev, m_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
    if ((rc = mm_load(ctx, dev, 0.0, (uint64_t)ctx->step_counter))) return rc;
    if ((rc = mm_advance(ctx, method, nsteps, dt_s, tol, 0.0, 0.0))) return rc;
    if ((rc = mm_store(ctx, dev))) return rc;
    CK(cudaMemcpyAsync(m_host, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MM_OK;
}

int mm_profile(mm_ctx* ctx, int enable) {
    if (!ctx) return MM_EINVAL;
    ctx->profiling = enable != 0;
    if (enable) {
        for (int i = 0; i < mm::NPASS; ++i) { ctx->pass_ms[i] = 0.0; ctx->pass_n[i] = 0; }
    }
    return MM_OK;
}

int mm_pass_times(mm_ctx* ctx, double* ms_out, long long* count_out) {
    if (!ctx) return MM_EINVAL;
    // every recorded pair is released, also when a query fails (the first error is returned)
    cudaError_t first = cudaStreamSynchronize(ctx->stream);
    for (auto& r : ctx->prof) {
        float ms = 0.f;
        const cudaError_t e = first == cudaSuccess ? cudaEventElapsedTime(&ms, r.a, r.b) : first;
        if (e == cudaSuccess) {
            ctx->pass_ms[r.pass] += ms;
            ctx->pass_n[r.pass] += 1;
        } else if (first == cudaSuccess) {
            first = e;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    ctx->prof.clear();
    if (first != cudaSuccess) return cuda_fail(ctx, first, "mm_pass_times");
    for (int i = 0; i < mm::NPASS; ++i) {
        if (ms_out) ms_out[i] = ctx->pass_ms[i];
        if (count_out) count_out[i] = ctx->pass_n[i];
    }
    return MM_OK;
}

const char* mm_last_error(const mm_ctx* ctx) {
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

void mm_destroy(mm_ctx* ctx) {
    if (!ctx) return;
    if (ctx->step_graph) cudaGraphExecDestroy(ctx->step_graph);
    for (auto& r : ctx->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    delete ctx;
}

int mm_eval_heff_static(mm_ctx* ctx, const float* m, float* h_out, float* torque_out) {
    if (!ctx) return MM_EINVAL;
    if (!ctx->have_material) return fail(ctx, MM_ESTATE, "material not set (mm_set_material)");
    if (ctx->demag && !ctx->kernel_ready)
        return fail(ctx, MM_ESTATE, "demag kernel not built (mm_demag_kernel) or demag not disabled");
    if (!m) return fail(ctx, MM_EINVAL, "null m");
    const size_t off_tw = align256(sizeof(mm::DevState));
    const size_t off_s1 = off_tw + align256((size_t)mmfft::TWN * sizeof(float2));
    const size_t off_s2 = off_s1 + align256(ctx->sz_s1);
    const size_t need = ctx->demag ? off_s2 + align256(ctx->sz_s2) : off_s1;    // no spectra without demag
    if (need > (size_t)MM_STATIC_SCRATCH_BYTES) {
        char buf[200];
        std::snprintf(buf, sizeof(buf),
                      "grid needs %zu bytes of scratch; the static scratch of mm_eval_heff_static holds %zu bytes "
                      "(MM_STATIC_SCRATCH_BYTES): use mm_eval_heff with a workspace", need,
                      (size_t)MM_STATIC_SCRATCH_BYTES);
        return fail(ctx, MM_ENOMEM, buf);
    }
    char* base = nullptr;
    int rc = static_scratch_for_current_device(ctx, &base);
    if (rc) return rc;
    const double tu = ctx->gamma0 * ctx->Ms;
    mm::HotParams p = hot_params(ctx, ctx->th_dt * tu, true);
    // everything the evaluation writes besides its outputs lives in the static array
    p.st = reinterpret_cast<mm::DevState*>(base);
    p.tw = reinterpret_cast<const float2*>(base + off_tw);
    p.s1 = reinterpret_cast<float2*>(base + off_s1);
    p.s2 = reinterpret_cast<float2*>(base + off_s2);
    p.kt = ctx->demag ? reinterpret_cast<const float*>(ctx->ws + ctx->off_kt) : nullptr;
    for (int i = 0; i < 2; ++i) { p.ms[i] = nullptr; p.ks[i] = nullptr; p.mstage[i] = nullptr; }
    for (int j = 0; j < 8; ++j) p.kb[j] = nullptr;
    p.hbuf = nullptr;
    p.zsplit = 0;                 // the FP32 z pass: its buffers stay in the static array
    p.m_eval = m;
    p.h_out = h_out;
    p.tq_out = torque_out;
    p.want_energy = 0;
    p.thermal_step = (long long)ctx->th_step;
    // the reduction counters must start at zero; the spectra are fully rewritten
    CK(cudaMemsetAsync(base, 0, sizeof(mm::DevState), ctx->stream));
    mm::LaunchArgs a{mm::SRC_PTR, mm::LM_EVAL, 0, 0, 0};
    int ids[8];
    const int n = mm::eval_passes(p, a, ids);
    for (int i = 0; i < n; ++i) CK(mm::launch_pass(p, a, ids[i], ctx->stream));
    return MM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched ensembles of independent samples (mm_batch_*).  Each sample keeps
// its own context (geometry, material, workspace slice, demag kernel, device
// state); a batch launches every pass once per FFT length over all samples
// of that length and replays one batched step from a CUDA graph.  Samples
// that reach their torque bound drop out of the launches (the work lists are
// rebuilt for the rest).
struct mm_batch {
    std::vector<mm_ctx*> ctx;                 // not owned
    cudaStream_t stream = nullptr;
    char* ws = nullptr;
    size_t ws_size = 0;
    size_t off_ps = 0, off_work = 0, off_states = 0, off_active = 0, total = 0;
    std::vector<mm::HotParams> hp_dev;        // what the device descriptors hold (uploaded on change)
    size_t max_work = 0;                      // int4 entries for all samples (both tile shapes, and a group's
                                              // alternative list while the autotuner times it)
    size_t work_used = 0;                     // entries of the current lists
    std::vector<int4> work_host;              // their host copy
    std::vector<mm::HotParams> hp;            // host copies of the device descriptors
    std::vector<int> active;                  // samples in the current work lists
    struct Group { int pass, logp, nb; size_t off; int variant; };
    std::vector<Group> groups;
    int tune_mode = 1;                        // 0 default kernels, 1 autotune, 2 alternative budget everywhere
    bool groups_ready = false;
    bool loaded = false;
    bool k1_valid = false;
    bool spec_m2 = false;                     // x spectrum of every sample holds m_2
    bool h_set = false;
    cudaGraphExec_t graph = nullptr;
    int graph_method = 0;
    std::string err;
};

namespace {

constexpr int kBatchPasses[] = {mm::PASS_XFWD, mm::PASS_YCONV, mm::PASS_YFWD, mm::PASS_ZCONV, mm::PASS_YINV,
                                mm::PASS_YZCONV, mm::PASS_XINV_H, mm::PASS_LOCAL_H, mm::PASS_XFWD_NEXT};

int bfail(mm_batch* b, int code, const std::string& msg) {
    if (b) b->err = msg;
    return code;
}

#define BCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return bfail(b, MM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// tile variant of a group (pass, FFT length) in the work lists: 2 = the half
// tile of the register x passes, else 0 (the register budgets share a list)
using TileMap = std::map<std::pair<int, int>, int>;

// blocks of every pass for the samples in `which` (work entries appended to out)
int batch_work(mm_batch* b, const std::vector<int>& which, std::vector<int4>* out,
               std::vector<mm_batch::Group>* groups, const TileMap* tiles = nullptr) {
    for (int pass : kBatchPasses) {
        // samples grouped by the pass's kernel (its FFT length; for the fused
        // y-z pass the length and the z cells per block)
        std::map<int, std::vector<int4>> by_logp;
        for (int i : which) {
            int gx = 0, gy = 0;
            int tile = 0;
            if (tiles) {
                auto it = tiles->find({pass, mm::batch_pass_logp(b->hp[i], pass)});
                if (it != tiles->end()) tile = it->second;
            }
            BCK(mm::batch_pass_grid(b->hp[i], pass, tile, &gx, &gy));
            const int nblk = gx * gy;
            if (nblk == 0) continue;
            const int lp = mm::batch_pass_logp(b->hp[i], pass);
            for (int by = 0; by < gy; ++by)
                for (int bx = 0; bx < gx; ++bx) by_logp[lp].push_back(make_int4(i, bx, by, nblk));
        }
        for (auto& kv : by_logp) {
            int tile = 0;
            if (tiles) {
                auto it = tiles->find({pass, kv.first});
                if (it != tiles->end()) tile = it->second;
            }
            if (groups) groups->push_back({pass, kv.first, (int)kv.second.size(), out->size(), tile});
            out->insert(out->end(), kv.second.begin(), kv.second.end());
        }
    }
    return MM_OK;
}

// Autotuner: each batched FFT pass is compiled with two register budgets
// (mm::batch_variants); for every group (pass, FFT length) whose budgets
// differ, time both on the loaded samples and keep the faster.  Choices are
// cached for the process, keyed by pass, FFT length and the power of two of
// the group's block count.  The timing launches run in evaluation mode and
// write only scratch (spectra, H_demag), which the next k1 pass rewrites.
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int>, int> g_tune_cache;

// destroys the timing events on every return path
struct EventPair {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~EventPair() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// Times every compiled variant of every group with more than one (the
// register budgets on the group's work list, the half tile of the register x
// passes on its own list, uploaded past the current lists) and records the
// fastest in *pick; a choice cached for the process is taken without timing.
int batch_tune(mm_batch* b, size_t work_used, std::map<size_t, int>* pick) {
    if (b->tune_mode == 0 || b->active.empty()) return MM_OK;
    const mm::LaunchArgs a = make_args(b->hp[b->active[0]], mm::SRC_CUR, mm::LM_EVAL, 0, false, false);
    const mm::HotParams* ps = reinterpret_cast<const mm::HotParams*>(b->ws + b->off_ps);
    int4* work = reinterpret_cast<int4*>(b->ws + b->off_work);
    EventPair ev;
    cudaEvent_t& e0 = ev.e0;
    cudaEvent_t& e1 = ev.e1;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const auto& g = b->groups[gi];
        const int nv = mm::batch_variants(g.pass, g.logp);
        if (nv < 2) continue;
        if (b->tune_mode == 2) { (*pick)[gi] = 1; continue; }
        if (b->tune_mode == 3) { (*pick)[gi] = nv >= 3 ? 2 : 0; continue; }
        const auto key = std::make_tuple(g.pass, g.logp, ilog2(g.nb));
        {
            std::lock_guard<std::mutex> lock(g_tune_mutex);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) { (*pick)[gi] = it->second; continue; }
        }
        if (!e0) { BCK(cudaEventCreate(&e0)); BCK(cudaEventCreate(&e1)); }
        float best = 0.f;
        int choice = 0;
        for (int v = 0; v < nv; ++v) {
            const int4* wv = work + g.off;
            int nb = g.nb;
            if (v == 2) {
                // this group's samples with the half tile, past the current lists
                std::vector<int> samples;
                int last = -1;
                for (size_t k = g.off; k < g.off + (size_t)g.nb && k < b->work_host.size(); ++k)
                    if (b->work_host[k].x != last) { samples.push_back(b->work_host[k].x); last = b->work_host[k].x; }
                TileMap one = {{{g.pass, g.logp}, 2}};
                std::vector<int4> alt;
                std::vector<mm_batch::Group> agroups;
                int rc = batch_work(b, samples, &alt, &agroups, &one);
                if (rc) return rc;
                size_t off = 0, cnt = 0;
                for (const auto& ag : agroups)
                    if (ag.pass == g.pass && ag.logp == g.logp) { off = ag.off; cnt = ag.nb; }
                if (cnt == 0 || work_used + cnt > b->max_work) continue;
                BCK(cudaMemcpyAsync(work + work_used, alt.data() + off, cnt * sizeof(int4), cudaMemcpyHostToDevice,
                                    b->stream));
                BCK(cudaStreamSynchronize(b->stream));
                wv = work + work_used;
                nb = (int)cnt;
            }
            BCK(mm::launch_pass_batched(ps, wv, nb, a, g.pass, g.logp, v, b->stream));   // warm-up
            BCK(cudaEventRecord(e0, b->stream));
            for (int r = 0; r < 3; ++r) BCK(mm::launch_pass_batched(ps, wv, nb, a, g.pass, g.logp, v, b->stream));
            BCK(cudaEventRecord(e1, b->stream));
            BCK(cudaEventSynchronize(e1));
            float ms = 0.f;
            BCK(cudaEventElapsedTime(&ms, e0, e1));
            if (v == 0 || ms < best) { best = ms; choice = v; }
        }
        (*pick)[gi] = choice;
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = choice;
    }
    return MM_OK;
}

// work lists for the active samples, uploaded to the batch workspace; then
// the autotuner's choices, and the lists again where it chose a tile shape
int batch_upload(mm_batch* b, const TileMap* tiles) {
    std::vector<int4> work;
    std::vector<mm_batch::Group> groups;
    int rc = batch_work(b, b->active, &work, &groups, tiles);
    if (rc) return rc;
    if (work.size() > b->max_work) return bfail(b, MM_ENOMEM, "batch work list larger than its reservation");
    if (!work.empty())
        BCK(cudaMemcpyAsync(b->ws + b->off_work, work.data(), work.size() * sizeof(int4), cudaMemcpyHostToDevice,
                            b->stream));
    BCK(cudaStreamSynchronize(b->stream));    // the host vector goes out of scope
    b->groups = groups;
    b->work_used = work.size();
    b->work_host.swap(work);
    return MM_OK;
}

int batch_build_groups(mm_batch* b) {
    int rc = batch_upload(b, nullptr);
    if (rc) return rc;
    if (!b->active.empty())
        BCK(cudaMemcpyAsync(b->ws + b->off_active, b->active.data(), b->active.size() * sizeof(int),
                            cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    std::map<size_t, int> pick;
    if ((rc = batch_tune(b, b->work_used, &pick))) return rc;
    TileMap tiles;
    for (const auto& kv : pick)
        if (kv.second == 2) tiles[{b->groups[kv.first].pass, b->groups[kv.first].logp}] = 2;
    std::map<std::pair<int, int>, int> budget;      // register budget of the groups that keep their tile
    for (const auto& kv : pick)
        if (kv.second != 2) budget[{b->groups[kv.first].pass, b->groups[kv.first].logp}] = kv.second;
    if (!tiles.empty() && (rc = batch_upload(b, &tiles))) return rc;
    for (auto& g : b->groups) {
        auto it = budget.find({g.pass, g.logp});
        if (g.variant != 2 && it != budget.end()) g.variant = it->second;
    }
    b->groups_ready = true;
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    return MM_OK;
}

int batch_eval(mm_batch* b, int src, int mode, int stage, bool fuse, bool have_spectrum) {
    const mm::LaunchArgs a = make_args(b->hp[b->active[0]], src, mode, stage, fuse, have_spectrum);
    const mm::HotParams* ps = reinterpret_cast<const mm::HotParams*>(b->ws + b->off_ps);
    const int4* work = reinterpret_cast<const int4*>(b->ws + b->off_work);
    for (const auto& g : b->groups) {
        if (g.pass == mm::PASS_XFWD && have_spectrum) continue;
        if (g.pass == mm::PASS_XFWD_NEXT && !fuse) continue;
        BCK(mm::launch_pass_batched(ps, work + g.off, g.nb, a, g.pass, g.logp, g.variant, b->stream));
    }
    return MM_OK;
}

// the launches of one batched Runge-Kutta step (as enqueue_step)
int batch_step(mm_batch* b, const RkInfo& r, bool first) {
    int rc;
    const int S = r.stages;
    auto src_of = [&](int st) { return (st & 1) ? mm::SRC_STAGE1 : mm::SRC_STAGE0; };
    if (r.fsal) {
        if ((rc = batch_eval(b, mm::SRC_COMBINE2, mm::LM_RK, 2, true, first))) return rc;
        for (int st = 3; st < S; ++st)
            if ((rc = batch_eval(b, src_of(st), mm::LM_RK, st, true, true))) return rc;
        return batch_eval(b, mm::SRC_NEXT, mm::LM_RKFINAL, S, false, true);
    }
    if ((rc = batch_eval(b, mm::SRC_CUR, mm::LM_K1, 1, true, false))) return rc;
    for (int st = 2; st < S; ++st)
        if ((rc = batch_eval(b, src_of(st), mm::LM_RK, st, true, true))) return rc;
    return batch_eval(b, src_of(S), mm::LM_RKFINAL, S, false, true);
}

// nsteps Runge-Kutta steps of the active samples.  dt_s > 0 sets every
// sample's step size (s); tol < 0 keeps it fixed.
int batch_advance(mm_batch* b, int method, long nsteps, double dt_s, double tol, double torque_tol) {
    RkInfo r;
    if (!rk_info(method, &r)) return bfail(b, MM_EINVAL, "batches run the Runge-Kutta methods (RK3 ... RKDP)");
    if (!b->loaded) return bfail(b, MM_ESTATE, "no state loaded (mm_batch_load)");
    if (b->active.empty() || nsteps <= 0) return MM_OK;
    const bool fixed_steps = !r.adaptive || tol < 0.0;
    if (r.adaptive && !fixed_steps && tol == 0.0) return bfail(b, MM_EINVAL, "adaptive methods need tol > 0");
    if (fixed_steps && !(dt_s > 0) && !b->h_set) return bfail(b, MM_EINVAL, "fixed steps need dt > 0");
    for (int i : b->active)        // checked before any sample's descriptor changes
        if (b->ctx[i]->T > 0.0) return bfail(b, MM_EINVAL, "batches run without the thermal field (temperature 0)");
    if (method != b->graph_method && b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    if (!b->groups_ready) {
        int rc = batch_build_groups(b);
        if (rc) return rc;
    }
    double dt0 = dt_s;
    if (!(dt0 > 0) && !b->h_set) dt0 = 1e-13;        // default first step 100 fs
    for (int i : b->active) {
        mm_ctx* c = b->ctx[i];
        mm::HotParams& p = b->hp[i];
        p = hot_params(c, 0.0, true);       // the step lives in each sample's device state
        p.rk = r.index;
        p.rk_stages = r.stages;
        p.rk_fsal = r.fsal;
        c->spec = mm_ctx::SPEC_NONE;               // single-context calls start afresh after a batch
        c->k1_valid = false;
    }
    if (dt0 > 0) b->h_set = true;
    // sample descriptors: copied only when they changed (a copy from pageable
    // memory waits for the stream); then one launch sets every active
    // sample's run parameters
    if (b->hp_dev.size() != b->hp.size() ||
        std::memcmp(b->hp_dev.data(), b->hp.data(), b->hp.size() * sizeof(mm::HotParams)) != 0) {
        BCK(cudaMemcpyAsync(b->ws + b->off_ps, b->hp.data(), b->hp.size() * sizeof(mm::HotParams),
                            cudaMemcpyHostToDevice, b->stream));
        b->hp_dev = b->hp;
    }
    BCK(mm::launch_set_run_batch(reinterpret_cast<const mm::HotParams*>(b->ws + b->off_ps),
                                 reinterpret_cast<const int*>(b->ws + b->off_active), (int)b->active.size(),
                                 fixed_steps ? 1.0 : tol, torque_tol > 0 ? torque_tol : 0.0, dt0 > 0 ? dt0 : 0.0,
                                 fixed_steps ? 1 : 0, b->stream));
    int rc;
    if (r.fsal) {
        if (dt_s > 0) b->spec_m2 = false;          // m_2 depends on h
        if (!b->k1_valid) {
            // k1 = f(m_n) for every sample; the same passes form m_2 and its spectrum
            if ((rc = batch_eval(b, mm::SRC_CUR, mm::LM_K1, 1, true, false))) return rc;
            b->k1_valid = true;
            b->spec_m2 = true;
        }
    }
    long s = 0;
    if (r.fsal && b->spec_m2) {
        if ((rc = batch_step(b, r, true))) return rc;
        b->spec_m2 = false;
        ++s;
    }
    if (s < nsteps) {
        if (!b->graph) {
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const int erc = batch_step(b, r, false);
                const cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
                if (erc == MM_OK && ee == cudaSuccess && g && cudaGraphInstantiate(&b->graph, g, 0) == cudaSuccess)
                    b->graph_method = method;
                else
                    b->graph = nullptr;
                if (g) cudaGraphDestroy(g);
            }
            cudaGetLastError();
        }
        for (; s < nsteps; ++s) {
            if (b->graph) BCK(cudaGraphLaunch(b->graph, b->stream));
            else if ((rc = batch_step(b, r, false))) return rc;
        }
    }
    if (!r.fsal) b->k1_valid = false;
    return MM_OK;
}

int batch_states(mm_batch* b, std::vector<mm::DevState>* out) {
    const int n = (int)b->ctx.size();
    out->resize(n);
    mm::DevState* d = reinterpret_cast<mm::DevState*>(b->ws + b->off_states);
    BCK(mm::launch_gather_states(reinterpret_cast<const mm::HotParams*>(b->ws + b->off_ps), d, n, b->stream));
    BCK(cudaMemcpyAsync(out->data(), d, n * sizeof(mm::DevState), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return MM_OK;
}

void fill_stats(mm_ctx* c, const mm::DevState& h, int method, mm_stats* s) {
    const double tu = c->gamma0 * c->Ms;
    s->evals = h.evals;
    s->accepted = h.accepted;
    s->rejected = h.rejected;
    s->step_index = h.step_index;
    s->t = h.t / tu;
    s->dt = h.h / tu;
    (void)method;
    s->last_err = h.last_err;
    s->max_torque = h.max_torque;
    const double V = c->dx * c->dy * c->dz;
    s->energy = MU0 * c->Ms * c->Ms * V * h.energy_acc;
    s->dissipation = -MU0 * c->Ms * c->Ms * c->Ms * V * c->gamma0 * c->alpha / (1.0 + c->alpha * c->alpha) *
                     h.tsq_acc;
    s->status = h.status;
    s->done = h.done;
}

}  // namespace

extern "C" {

int mm_batch_create(mm_batch** out, mm_ctx* const* ctxs, int n, void* cuda_stream) {
    if (!out) return MM_EINVAL;
    *out = nullptr;
    if (!ctxs || n < 1) return MM_EINVAL;
    mm_batch* b = new (std::nothrow) mm_batch();
    if (!b) return MM_ENOMEM;
    b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    b->ctx.assign(ctxs, ctxs + n);
    b->hp.resize(n);
    for (int i = 0; i < n; ++i) {
        mm_ctx* c = ctxs[i];
        if (!c || check_ready(c, true) != MM_OK || !c->demag) {
            delete b;
            return MM_EINVAL;
        }
        b->hp[i] = hot_params(c, 0.0, false);
        b->hp[i].rk_stages = 7;
        if (!mm::batch_supported(b->hp[i])) {
            delete b;
            return MM_EINVAL;
        }
    }
    std::vector<int> all(n);
    for (int i = 0; i < n; ++i) all[i] = i;
    std::vector<int4> work, half;
    TileMap all_half;
    for (int pass : kBatchPasses)
        for (int i = 0; i < n; ++i) {
            const int lp = mm::batch_pass_logp(b->hp[i], pass);
            if (mm::batch_variants(pass, lp) >= 3) all_half[{pass, lp}] = 2;
        }
    if (batch_work(b, all, &work, nullptr) != MM_OK || batch_work(b, all, &half, nullptr, &all_half) != MM_OK) {
        delete b;
        return MM_EINVAL;
    }
    // the longer of the two lists, plus room for one group's alternative list
    b->max_work = std::max(work.size(), half.size()) + half.size();
    for (int i = 0; i < n; ++i) ctxs[i]->stream = b->stream;    // every sample's work goes on the batch stream
    size_t off = 0;
    b->off_ps = off; off += align256((size_t)n * sizeof(mm::HotParams));
    b->off_work = off; off += align256(b->max_work * sizeof(int4));
    b->off_states = off; off += align256((size_t)n * sizeof(mm::DevState));
    b->off_active = off; off += align256((size_t)n * sizeof(int));
    b->total = off;
    b->active = all;
    *out = b;
    return MM_OK;
}

size_t mm_batch_workspace_bytes(const mm_batch* b) { return b ? b->total : 0; }

int mm_batch_set_workspace(mm_batch* b, void* dev_ptr, size_t bytes) {
    if (!b || !dev_ptr) return bfail(b, MM_EINVAL, "null workspace");
    if (reinterpret_cast<uintptr_t>(dev_ptr) & 255) return bfail(b, MM_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < b->total) return bfail(b, MM_ENOMEM, "workspace smaller than mm_batch_workspace_bytes()");
    b->ws = static_cast<char*>(dev_ptr);
    b->ws_size = bytes;
    b->groups_ready = false;
    b->hp_dev.clear();
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    BCK(cudaMemcpyAsync(b->ws + b->off_ps, b->hp.data(), b->hp.size() * sizeof(mm::HotParams),
                        cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    b->hp_dev = b->hp;
    return MM_OK;
}

int mm_batch_load(mm_batch* b, const float* const* m) {
    if (!b || !m) return MM_EINVAL;
    if (!b->ws) return bfail(b, MM_ENOMEM, "workspace not set (mm_batch_set_workspace)");
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        const int rc = mm_load(b->ctx[i], m[i], 0.0, 0);
        if (rc) return bfail(b, rc, "sample " + std::to_string(i) + ": " + b->ctx[i]->err);
    }
    std::vector<int> all(b->ctx.size());
    for (size_t i = 0; i < all.size(); ++i) all[i] = (int)i;
    if (b->active != all || !b->groups_ready) {
        b->active = all;
        b->groups_ready = false;
    }
    b->loaded = true;
    b->k1_valid = false;
    b->spec_m2 = false;
    b->h_set = false;
    return MM_OK;
}

int mm_batch_store(mm_batch* b, float* const* m) {
    if (!b || !m) return MM_EINVAL;
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        const int rc = mm_store(b->ctx[i], m[i]);
        if (rc) return bfail(b, rc, "sample " + std::to_string(i) + ": " + b->ctx[i]->err);
    }
    return MM_OK;
}

int mm_batch_advance(mm_batch* b, int method, long nsteps, double dt_s, double tol) {
    if (!b) return MM_EINVAL;
    if (!b->ws) return bfail(b, MM_ENOMEM, "workspace not set (mm_batch_set_workspace)");
    if (nsteps < 0 || !std::isfinite(dt_s) || !std::isfinite(tol)) return bfail(b, MM_EINVAL, "bad arguments");
    return batch_advance(b, method, nsteps, dt_s, tol, 0.0);
}

int mm_batch_get_stats(mm_batch* b, mm_stats* out) {
    if (!b || !out) return MM_EINVAL;
    if (!b->ws) return bfail(b, MM_ENOMEM, "workspace not set");
    std::vector<mm::DevState> h;
    int rc = batch_states(b, &h);
    if (rc) return rc;
    for (size_t i = 0; i < b->ctx.size(); ++i) fill_stats(b->ctx[i], h[i], b->graph_method, &out[i]);
    return MM_OK;
}

int mm_batch_relax(mm_batch* b, float* const* m, double torque_tol, double err_tol, long max_steps,
                   long* steps_out, double* torque_out, int* n_converged) {
    if (!b || !m) return MM_EINVAL;
    if (!(torque_tol > 0) || !(err_tol > 0) || max_steps < 0) return bfail(b, MM_EINVAL, "bad relax arguments");
    int rc = mm_batch_load(b, m);
    if (rc) return rc;
    const int n = (int)b->ctx.size();
    std::vector<mm::DevState> h;
    std::vector<char> finished(n, 0);
    long done_steps = 0;
    bool first = true;
    while (true) {
        const long chunk = (max_steps - done_steps) < 64 ? (max_steps - done_steps) : 64;
        if ((rc = batch_advance(b, MM_RKDP, chunk, first ? 1e-13 : 0.0, err_tol, torque_tol))) return rc;
        first = false;
        done_steps += chunk;
        if ((rc = batch_states(b, &h))) return rc;
        std::vector<int> still;
        for (int i : b->active) {
            if (h[i].status) return bfail(b, h[i].status, "sample " + std::to_string(i) + " failed on the device");
            if (h[i].done) finished[i] = 1;
            else still.push_back(i);
        }
        if (still.empty() || done_steps >= max_steps) break;
        if (still.size() != b->active.size()) {
            b->active = still;                       // finished samples leave the launches
            if ((rc = batch_build_groups(b))) return rc;
        }
    }
    if ((rc = mm_batch_store(b, m))) return rc;
    BCK(cudaStreamSynchronize(b->stream));
    int conv = 0;
    for (int i = 0; i < n; ++i) {
        const bool ok = finished[i] && h[i].max_torque < torque_tol;
        conv += ok;
        if (steps_out) steps_out[i] = (long)(h[i].accepted + h[i].rejected);
        if (torque_out) torque_out[i] = h[i].max_torque;
    }
    if (n_converged) *n_converged = conv;
    // the next call starts from every sample again
    std::vector<int> all(n);
    for (int i = 0; i < n; ++i) all[i] = i;
    b->active = all;
    b->groups_ready = false;
    if (conv < n) return bfail(b, MM_ENOTCONVERGED, std::to_string(n - conv) + " samples did not reach the torque bound");
    return MM_OK;
}

int mm_batch_set_tuning(mm_batch* b, int mode) {
    if (!b) return MM_EINVAL;
    if (mode < 0 || mode > 3) return bfail(b, MM_EINVAL, "tuning mode must be 0, 1, 2 or 3");
    if (mode != b->tune_mode) {
        b->tune_mode = mode;
        b->groups_ready = false;                     // chosen again at the next advance
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    }
    return MM_OK;
}

int mm_batch_tuning(const mm_batch* b, int* n_groups, int* n_tunable, int* n_alternative) {
    if (!b) return MM_EINVAL;
    int g = 0, t = 0, alt = 0;
    for (const auto& gr : b->groups) {
        ++g;
        t += mm::batch_variants(gr.pass, gr.logp) > 1;
        alt += gr.variant != 0;
    }
    if (n_groups) *n_groups = g;
    if (n_tunable) *n_tunable = t;
    if (n_alternative) *n_alternative = alt;
    return MM_OK;
}

const char* mm_batch_last_error(const mm_batch* b) {
    if (!b) return "null batch";
    return b->err.c_str();
}

void mm_batch_destroy(mm_batch* b) {
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    delete b;
}

}  // extern "C"
