// hotpath_odd_yz.cu - the y and z passes of the FFT lengths R0 * 2^a with an
// odd factor R0 = 3, 5 or 7 (the sizes 2^n {1,3,5,7} of Sec. 3.3): the column
// pass with the kernel product (2-D y lines, 3-D z lines) and the 3-D y
// passes, all with their lines in shared memory.
#include "hotpath_kernels.cuh"

namespace mm {

#define MM_ODD_YZ_LENGTHS(X) X(3, 6) X(3, 7) X(3, 8) X(3, 9) X(3, 10) X(5, 6) X(5, 7) X(5, 8) X(5, 9) \
    X(7, 6) X(7, 7) X(7, 8) X(7, 9)

template <int R0, int L>
static void launch_yz_odd(const HotParams& p, const LaunchArgs& a, int pass, cudaStream_t s) {
    using S = OS<L, R0>;
    const size_t smc = (size_t)S::NL * S::LS * sizeof(float2), smy = (size_t)S::NLY * S::LS * sizeof(float2);
    switch (pass) {
        case PASS_YCONV:
            k_colconv_odd<L, R0, 0><<<(p.hx + S::COLS - 1) / S::COLS, S::NT, smc, s>>>(p, a);
            break;
        case PASS_ZCONV:
            k_colconv_odd<L, R0, 1><<<dim3(p.hx, (p.py + S::COLS - 1) / S::COLS), S::NT, smc, s>>>(p, a);
            break;
        case PASS_YFWD:
            k_ypass_odd<L, R0, false><<<dim3(p.hx, (p.nz + S::TZ - 1) / S::TZ), S::NTY, smy, s>>>(p, a);
            break;
        default:
            k_ypass_odd<L, R0, true><<<dim3(p.hx, (p.nz + S::TZ - 1) / S::TZ), S::NTY, smy, s>>>(p, a);
            break;
    }
}

cudaError_t launch_yz_mixed(const HotParams& p, const LaunchArgs& a, int pass, cudaStream_t s) {
    if (pass != PASS_YCONV && pass != PASS_ZCONV && pass != PASS_YFWD && pass != PASS_YINV)
        return cudaErrorInvalidValue;
    const int r = pass == PASS_ZCONV ? p.rz : p.ry, l = pass == PASS_ZCONV ? p.logpz : p.logpy;
    switch (r * 100 + l) {
#define MM_CASE(R, L) case R * 100 + L: launch_yz_odd<R, L>(p, a, pass, s); break;
        MM_ODD_YZ_LENGTHS(MM_CASE)
#undef MM_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int R0, int L>
static cudaError_t set_attr_odd_yz() {
    cudaError_t e;
    const int mx = 200 * 1024;
    if ((e = cudaFuncSetAttribute(k_colconv_odd<L, R0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_colconv_odd<L, R0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_ypass_odd<L, R0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    return cudaFuncSetAttribute(k_ypass_odd<L, R0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

cudaError_t configure_odd_yz_kernels() {
    cudaError_t e = cudaSuccess;
#define MM_SET(R, L) if ((e = set_attr_odd_yz<R, L>())) return e;
    MM_ODD_YZ_LENGTHS(MM_SET)
#undef MM_SET
    return e;
}

bool odd_yz_length_supported(int r, int logp) {
    switch (r * 100 + logp) {
#define MM_OK_CASE(R, L) case R * 100 + L: return true;
        MM_ODD_YZ_LENGTHS(MM_OK_CASE)
#undef MM_OK_CASE
        default: return false;
    }
}

}  // namespace mm
