// k_reweight_static.cu -- msa_reweight_static: the sequence reweighting of
// msa_reweight without any allocation and without a context.
//
// Some callers cannot allocate device memory at the time they need the
// weights: code that runs while another component owns the allocator (for
// example inside a memory-pool or caching-allocator callback), programs
// that must not allocate after start-up (fixed-memory services, real-time
// pipelines), and callers that only hold a raw stream.  This entry point
// takes its scratch space from one file-scope device array instead of
// cudaMalloc, and never calls cudaMalloc, cudaFree, cudaMallocHost or any
// allocating library routine.
//
// The array, kScratchBytes = 16 MiB, is part of the library image: every
// GPU that loads the library holds it until the process exits.  All calls
// share it and it keeps the previous call's contents; the regions that must
// start at zero are cleared on the stream at the start of every call.  Two
// calls whose work overlaps on the GPU (different streams, or one device
// used from several host threads without ordering) race on the array and
// give undefined results: order them.
//
// In host code the array's name is a host-side stand-in, not a device
// address.  Every call looks the device address up again with
// cudaGetSymbolAddress, with the stream's device current (a host-side
// lookup, no allocation), so an address never outlives the context it
// belongs to: after cudaDeviceReset, or from another context on the same
// device, the next call gets the array of the context that is current.
// The first call in a context may load the library's device code; make it
// before any stream capture.
#include "../../include/plmdca.h"
#include "plm_internal.cuh"

namespace {

constexpr size_t kScratchBytes = 16u << 20;  // 16 MiB

// the shared scratch of every call on a device: bit-planes, counts,
// histogram and the state-range flag
__device__ __align__(256) unsigned char g_reweight_scratch[kScratchBytes];

// marks B_eff as NaN when some state was outside 0..20
__global__ void k_flag_to_beff(const int *err, double *beff)
{
    if (*err) *beff = __longlong_as_double(0x7FF8000000000000LL);
}

}  // namespace

extern "C" plm_status msa_reweight_static(const int8_t *msa, int B, int N, int q, double x,
                                          int32_t *m_out, float *w_out, double *beff_out,
                                          void *cuda_stream)
{
    if (q != plm::Q || B < 1 || N < 1 || !msa || !beff_out) return PLM_EINVAL;
    if (!(x >= 0.0 && x <= 1.0)) return PLM_EINVAL;

    // scratch needed: [planes | m | hist] as laid out by the reweighting
    // kernels, then the state-range flag
    const size_t rw = plm::reweight_scratch_bytes(B, N);
    const size_t need = rw + 256;
    if (need > kScratchBytes) return PLM_ENOMEM;  // beyond the static maximum

    // the work runs on the stream's device, which must be the current one:
    // the array's address below is the current device's
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PLM_ECUDA;
    }
    if (st) {
        int sdev = -1;
        if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
            cudaGetLastError();
            return PLM_EINVAL;
        }
        if (sdev != dev) return PLM_EINVAL;
    }
    void *base = nullptr;
    if (cudaGetSymbolAddress(&base, g_reweight_scratch) != cudaSuccess || !base) {
        cudaGetLastError();
        return PLM_ECUDA;
    }
    unsigned char *scratch = (unsigned char *)base;
    int *err = (int *)(scratch + rw);

    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) {
        cudaGetLastError();
        return PLM_ECUDA;
    }
    // the launcher clears the counts and the histogram itself
    cudaError_t e = plm::launch_reweight(msa, B, N, plm::identity_threshold(x, N), m_out, w_out,
                                         beff_out, scratch, err, st);
    if (e == cudaSuccess) {
        k_flag_to_beff<<<1, 1, 0, st>>>(err, beff_out);
        plm::count_launches(1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PLM_ECUDA;
    }
    return PLM_OK;
}
