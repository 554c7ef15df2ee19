// mm_internal.cuh - types shared by the CUDA translation units of libmm.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mm {

// Device-resident integrator state (lives in the caller's workspace).  All
// times are in internal units (1/(gamma0 Ms)); fields in units of Ms.
struct DevState {
    double t;             // simulated time
    double h;             // adaptive step (RKDP)
    double t_end;         // stop time (<= 0: none)
    double tol;           // RKDP error bound per step
    double torque_tol;    // relaxation target (<= 0: none)
    double h_min;         // smallest admissible step
    double last_err;      // last RKDP error estimate
    double max_torque;    // max |m x h| of the last accepted state
    double energy_acc;    // sum of energy densities (EVAL mode)
    double tsq_acc;       // sum of |m x h|^2 (EVAL mode), internal units
    double max_dm;        // > 0: fixed maximum variation of m per step (h set by the k1 pass)
    double h_cap;         // upper bound on that h (<= 0: none)
    unsigned long long kre_bits;  // max |Re K^| seen by the kernel setup (double bits)
    unsigned long long kim_bits;  // max |Im K^| seen by the kernel setup (double bits)
    long long step_index; // thermal clock (Euler/Heun)
    long long accepted;
    long long rejected;
    long long evals;
    unsigned int err_bits;     // atomicMax of non-negative float bits
    unsigned int torque_bits;  // atomicMax of non-negative float bits
    unsigned int blocks_done;  // last-block detection
    unsigned int bad;          // non-finite value seen
    int cur;              // which of the two state slots holds m_n / k1
    int after_reject;     // previous RKDP attempt was rejected
    int done;             // run finished (t_end, torque target, failure)
    int status;           // 0 or a negative mm_status
    int fixed_h;          // RKDP without step control: every step accepted, h kept
    int pad_;
};

// Local epilogue modes (what the inverse-x kernel does with H_eff and dm/dt).
enum LocalMode : int {
    LM_EVAL = 0,      // write H (A/m) and dm/dt (1/s); optional energy
    LM_K1 = 1,        // k1 = f(m_n) into the current k slot; torque check
    LM_RK = 2,        // Runge-Kutta stage s = 2..S-1: k_s and the input of stage s+1
    LM_RKFINAL = 3,   // last stage S: error, torque, (m_{n+1} without FSAL), step control
    LM_EULER = 4,
    LM_HEUN1 = 5,
    LM_HEUN2 = 6,
};

// Where an evaluation reads its magnetisation from.
enum Source : int {
    SRC_PTR = 0,      // HotParams::m_eval (user array)
    SRC_CUR = 1,      // state slot ms[cur]  (m_n)
    SRC_NEXT = 2,     // state slot ms[1-cur] (candidate m_{n+1})
    SRC_STAGE0 = 3,   // mstage[0]
    SRC_STAGE1 = 4,   // mstage[1]
    SRC_COMBINE2 = 5, // m_n + h a21 k1, also written to mstage[0]
};

struct HotParams {
    // geometry
    int nx, ny, nz;
    int px, py, pz;          // FFT lengths: r * 2^logp
    int logpx, logpy, logpz;
    int rx, ry, rz;          // odd factor of each FFT length (1, 3, 5 or 7)
    int hx;                  // px/2 + 1
    int hyk, hzk;            // stored kernel extents along y and z (P/2 + 1)
    int nyp;                 // y extent stored in the x-spectrum (multiple of 16)
    int nzp;                 // z extent stored in the y-spectrum (multiple of 8)
    int ty;                  // rows per block in the x kernels
    int tz;                  // z lines per block in the 3-D y kernels
    int tky;                 // ky lines per block in the 3-D z kernel
    int kxb;                 // kx columns per block in the 2-D y kernel
    int pbc[3];
    int ncomp;               // 4 (nz == 1) or 6 stored kernel components
    long long ncell;
    // material, internal units
    float cex[3];            // 2A/(mu0 Ms^2 d^2) per axis
    float kan;               // 2Ku/(mu0 Ms^2)
    float ux, uy, uz;        // easy axis
    const float* uaxis;      // per-cell unit easy axes [3][ncell] (caller-owned), or null: (ux, uy, uz)
    float hzx, hzy, hzz;     // B/(mu0 Ms)
    float kc1, kc2;          // cubic anisotropy 2K1/(mu0 Ms^2), 2K2/(mu0 Ms^2) (0: off)
    float c[3][3];           // orthonormal cubic axes c1, c2, c3
    float stt_s[3];          // spin-transfer torque: b_j j_a / (2 d_a gamma0 Ms) per axis (0: off)
    float stt_beta;          // xi - alpha
    int stt;                 // spin-transfer torque on
    float alpha;
    float llpref;            // 1/(1+alpha^2)
    float sigma_th;          // thermal sigma / Ms for the current dt (0: off)
    unsigned long long seed;
    long long thermal_step;  // EVAL-mode thermal clock
    int demag;
    int small_cl;            // > 0: each evaluation is one cluster launch of this many CTAs (hotpath_small.cu)
    // step (internal units)
    double dt_d;             // Euler/Heun fixed step
    int rk;                  // Runge-Kutta tableau index (hotpath.cu c_rka)
    int rk_stages;           // its number of stages
    int rk_fsal;             // its last stage evaluates the new solution
    // output scales
    float h_scale;           // Ms (A/m)
    float t_scale;           // gamma0 Ms (1/s)
    double t_unit;           // gamma0 Ms (1/s) in double: seconds -> internal time
    // buffers
    const float2* tw;
    const float2* twr[8];    // twr[r]: exp(-2 pi i t / (r TWN)), t < r TWN, for the odd factors r in use
    const float* kt;
    float2* s1;
    float2* s2;
    DevState* st;
    float* ms[2];
    float* ks[2];
    float* kb[8];            // k2..k6 at kb[2..6]
    float* mstage[2];
    float* hbuf;             // H_demag [3][ncell] between the inverse x pass and the cell pass
    const float* m_eval;
    float* h_out;
    float* tq_out;
    int want_energy;
    // split-BF16 tensor-core variant of the 3-D z column pass (split_dft.cu)
    int zsplit;              // 1: the z pass runs as DFT products on the tensor cores
    int zs_kp;               // 2 * nzp: real width of a z line (re, im interleaved)
    void* zs_a_hi;           // [3*hx*py][kp] bf16 lines of s2, hi and lo parts
    void* zs_a_lo;
    float* zs_x;             // [3*hx*py][2*pz] forward transform (fp32)
    void* zs_y_hi;           // [3*hx*py][2*pz] bf16 product with the kernel, hi and lo parts
    void* zs_y_lo;
    float* zs_o;             // [3*hx*py][kp] inverse transform (fp32)
    const void* zs_f_hi;     // [2*pz][kp] forward DFT matrix, hi and lo parts
    const void* zs_f_lo;
    const void* zs_g_hi;     // [kp][2*pz] inverse DFT matrix, hi and lo parts
    const void* zs_g_lo;
    unsigned* zs_err;        // error word of the tensor-core products
};

struct LaunchArgs {
    int src;                 // Source of the evaluation input
    int mode;                // LocalMode
    int stage;               // RK stage (2..7)
    int fuse = 0;            // inverse-x pass also transforms the next evaluation's input
    int have_spectrum = 0;   // s1 already holds the x spectrum of this evaluation's input
    int next_src = 0;        // Source of the next evaluation's input (transformed when fuse)
    int keep = 0;            // that transform runs even when the run has finished (Euler/Heun
                             // keep the spectrum of m_n in place between calls)
    unsigned need = 0;       // bit j: the cell pass reads k_j (stage_need_mask)
};

// passes of one evaluation (the kernels of hotpath.cu), in launch order
enum Pass : int {
    PASS_XFWD = 0, PASS_YCONV = 1, PASS_YFWD = 2, PASS_ZCONV = 3, PASS_YINV = 4,
    PASS_XINV_LOCAL = 5, PASS_COMBINE2 = 6, PASS_LOCAL = 7, PASS_XINV_FUSED = 8,
    PASS_XINV_H = 9,        // inverse x transform alone: H_demag into hbuf
    PASS_LOCAL_H = 10,      // cell pass with H_demag from hbuf
    PASS_XFWD_NEXT = 11,    // forward x transform of the next evaluation's input
    PASS_SMALL = 12,        // the whole evaluation in one cluster launch (small 2-D grids)
    PASS_YZCONV = 13,       // 3-D grids with nz <= 8: y forward, z column pass and y inverse in one pass
    NPASS = 14
};

// hot path (hotpath.cu)
cudaError_t launch_normalize_load(const HotParams& p, const float* m_user, cudaStream_t s);
cudaError_t launch_copy_out(const HotParams& p, float* m_user, cudaStream_t s);
cudaError_t launch_copy_in(const HotParams& p, const float* m_user, cudaStream_t s);
// Euler step with the h its k1 pass set (fixed maximum variation of m per step)
cudaError_t launch_euler_update(const HotParams& p, cudaStream_t s);
int eval_passes(const HotParams& p, const LaunchArgs& a, int* ids);     // fills <= 7 pass ids
cudaError_t launch_pass(const HotParams& p, const LaunchArgs& a, int pass, cudaStream_t s);
cudaError_t configure_hot_kernels();
unsigned stage_need_mask(int rk, int mode, int stage);   // host: which k_j a pass reads
bool odd_x_length_supported(int r, int logp);          // x length r * 2^logp has compiled passes (r = 3, 5, 7)
// the x passes of those lengths (hotpath_odd.cu)
cudaError_t launch_x_mixed(const HotParams& p, const LaunchArgs& a, int pass, cudaStream_t s);
cudaError_t configure_odd_kernels();
// the y and z passes of those lengths (hotpath_odd_yz.cu)
bool odd_yz_length_supported(int r, int logp);
cudaError_t launch_yz_mixed(const HotParams& p, const LaunchArgs& a, int pass, cudaStream_t s);
cudaError_t configure_odd_yz_kernels();

// one-launch evaluation of small 2-D grids (hotpath_small.cu): CTAs per
// cluster for this geometry (0: does not apply), the launch, the attributes
int small_cluster_size(const HotParams& p);
cudaError_t launch_small(const HotParams& p, const LaunchArgs& a, cudaStream_t s);
// a run of nsteps standard steps (the n evaluations of one step, in order) in one launch
struct SmallSteps {
    long long nsteps;
    int n;
    LaunchArgs a[8];
};
cudaError_t launch_small_steps(const HotParams& p, const SmallSteps& steps, cudaStream_t s);
cudaError_t configure_small_kernels();

// the y and z stages of 3-D grids with few z cells in one pass (hotpath_yz.cu):
// 4 or 8 z cells per block where it applies, else 0; its launches
int yz_fused_nz(const HotParams& p);
cudaError_t launch_yzconv(const HotParams& p, const LaunchArgs& a, cudaStream_t s);
cudaError_t launch_yzconv_batched(const HotParams* ps, const int4* work, int nb, const LaunchArgs& a, int code,
                                  cudaStream_t s);
cudaError_t configure_yz_kernels();

// batched passes over independent samples (hotpath.cu)
bool batch_supported(const HotParams& p);
int batch_pass_logp(const HotParams& p, int pass);
// blocks of a pass for one sample (variant 2 of the register x passes: the half tile)
cudaError_t batch_pass_grid(const HotParams& p, int pass, int variant, int* gx, int* gy);
cudaError_t launch_pass_batched(const HotParams* ps, const int4* work, int nb, const LaunchArgs& a, int pass,
                                int logp, int variant, cudaStream_t s);
int batch_variants(int pass, int logp);     // kernels compiled for this pass: register budgets, tile shapes
cudaError_t launch_gather_states(const HotParams* ps, DevState* out, int n, cudaStream_t s);
// run parameters of the active samples of a batch, one launch (as a per-context
// mm_advance would set them; dt0_s > 0 sets the step, in seconds)
cudaError_t launch_set_run_batch(const HotParams* ps, const int* active, int n_active, double tol,
                                 double torque_tol, double dt0_s, int fixed_h, cudaStream_t s);

// split-BF16 z pass (split_dft.cu): bytes of its buffers, its tables, its launches
size_t zsplit_bytes(int nx, int ny, int nz, int hx, int py, int pz, int nzp, size_t* sizes /*7*/);
cudaError_t zsplit_tables(const HotParams& p, cudaStream_t s);
cudaError_t launch_zconv_split(const HotParams& p, const LaunchArgs& a, cudaStream_t s);

// kernel setup (setup.cu)
struct SetupParams {
    int nx, ny, nz;
    int px, py, pz;
    int ox, oy, oz;          // octant extents of the real-space tensor
    int pbc[3];
    int images;
    int ncomp;
    int hx, hyk, hzk;
    double dx, dy, dz;       // cell edges scaled so that max edge = 1
    double gl_t[4][8];       // Gauss-Legendre nodes on [-1, 1] for the orders below
    double gl_w[4][8];
    int gl_n[4];             // node counts, increasing; gl_n[3] used nearest
    double* oct;             // [6][oz][oy][ox] FP64 tensor octant
    double2* work;           // px*py*pz complex FP64 scratch
    float* kt;               // [ncomp][hx][hyk][hzk] float32 result
    DevState* st;
};
cudaError_t launch_kernel_setup(const SetupParams& p, cudaStream_t s);

}  // namespace mm

namespace mm {
// tensor-core product (tc_gemm.cu): C[b] = alpha * A[b] B[b]^T (+ C[b] when beta),
// A [m][k], B [n][k] bf16 row-major (k contiguous), C [m][n] fp32 row-major;
// strides in elements.  *err gets a non-zero bit when a bounded wait ran out.
cudaError_t gemm_bf16(const void* a, long long lda, long long a_batch, const void* b, long long ldb,
                      long long b_batch, float* c, long long ldc, long long c_batch, int m, int n, int k, int batch,
                      float alpha, int beta, unsigned* err, cudaStream_t s);
cudaError_t gemm_configure();   // once per device, before any capture of a product
}  // namespace mm
