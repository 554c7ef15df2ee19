// hotpath_odd.cu - the x passes of the FFT lengths R0 * 2^a with an odd factor
// R0 = 3, 5 or 7 (the sizes 2^n {1,3,5,7} of Sec. 3.3), in a translation unit of
// their own so that the library's files compile in parallel.
#include "hotpath_kernels.cuh"

namespace mm {

// x lengths R0 * 2^L with an odd factor R0 (shared-memory passes only):
// 3 * 2^6 .. 3 * 2^10, 5 * 2^6 .. 5 * 2^9, 7 * 2^6 .. 7 * 2^9
#define MM_ODD_X_LENGTHS(X) X(3, 6) X(3, 7) X(3, 8) X(3, 9) X(3, 10) X(5, 6) X(5, 7) X(5, 8) X(5, 9) \
    X(7, 6) X(7, 7) X(7, 8) X(7, 9)
template <int R0, int L>
static void launch_x_odd(const HotParams& p, const LaunchArgs& a, int pass, cudaStream_t s) {
    using S = XS<L, R0>;
    const dim3 g((p.ny + S::TY - 1) / S::TY, p.nz);
    const size_t sm = (size_t)S::NL * S::LS * sizeof(float2);
    if (pass == PASS_XFWD) { k_xfwd<L, R0><<<g, S::NT, sm, s>>>(p, a); return; }
    if (pass == PASS_XINV_LOCAL) k_xinv_local<L, false, false, R0><<<g, S::NT, sm, s>>>(p, a);
    else k_xinv_local<L, true, false, R0><<<g, S::NT, sm, s>>>(p, a);
}
cudaError_t launch_x_mixed(const HotParams& p, const LaunchArgs& a, int pass, cudaStream_t s) {
    if (pass != PASS_XFWD && pass != PASS_XINV_LOCAL && pass != PASS_XINV_FUSED) return cudaErrorInvalidValue;
    switch (p.rx * 100 + p.logpx) {
#define MM_CASE(R, L) case R * 100 + L: launch_x_odd<R, L>(p, a, pass, s); break;
        MM_ODD_X_LENGTHS(MM_CASE)
#undef MM_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}
template <int R0, int L>
static cudaError_t set_attr_odd_x() {
    cudaError_t e;
    const int mx = 200 * 1024;
    if ((e = cudaFuncSetAttribute(k_xfwd<L, R0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_xinv_local<L, false, false, R0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)))
        return e;
    return cudaFuncSetAttribute(k_xinv_local<L, true, false, R0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}
cudaError_t configure_odd_kernels() {
    cudaError_t e = cudaSuccess;
#define MM_SET(R, L) if ((e = set_attr_odd_x<R, L>())) return e;
    MM_ODD_X_LENGTHS(MM_SET)
#undef MM_SET
    return e;
}
bool odd_x_length_supported(int r, int logp) {
    switch (r * 100 + logp) {
#define MM_OK_CASE(R, L) case R * 100 + L: return true;
        MM_ODD_X_LENGTHS(MM_OK_CASE)
#undef MM_OK_CASE
        default: return false;
    }
}


}  // namespace mm
