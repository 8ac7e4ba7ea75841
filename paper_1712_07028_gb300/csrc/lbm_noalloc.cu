// lbm_noalloc.cu -- bubble volumes without any device allocation.
//
// Some callers cannot call cudaMalloc: code running where allocation is forbidden or
// deferred (inside an allocator hook, a signal-safe or real-time section, a host callback),
// or a host program whose memory budget is fixed and fully handed out before it starts.
// lbm_bubble_volumes_noalloc serves them: the bubble-volume sums of lbm_step's bubble model,
// per bubble id, whose scratch (per-id partial sums) is a file-scope static device array, so
// the call itself allocates nothing.  The caller still passes its inputs and the output.
#include <cstdio>
#include <mutex>

#include "lbm_internal.cuh"

namespace {

constexpr int kNoallocMaxBubbles = 1024;   // 1024 x 16 B of static scratch per device
constexpr int kNoallocMaxDevices = 64;

// scratch: [0, max) interface part of V_b (FP64), [max, 2 max) gas-cell counts (as uint64)
static __device__ __align__(256) unsigned long long g_bubble_scratch[2 * kNoallocMaxBubbles];

std::mutex g_setup_mutex;
struct DeviceSetup {
    unsigned long long* scratch;   // device address of g_bubble_scratch on this device
    int sms;                       // its multiprocessor count (grid size of the reduction)
};
DeviceSetup g_setup[kNoallocMaxDevices] = {};

// Per bubble id b: V_b = #gas cells carrying id b + sum over the interface cells carrying id b
// of (1 - phi), FP64, from canonical inputs (types LBM_CELL_*, owner -1 for none) -- the two
// sums the step's bubble model keeps per id.  Cells keep the id they were created with, so the
// volume of a merged bubble is the sum of these per-id volumes over its ids (one root).
__global__ void bubble_volumes_static_kernel(const uint8_t* __restrict__ flags, const int32_t* __restrict__ owner,
                                             const float* __restrict__ phi, size_t n, int nbub,
                                             unsigned long long* scratch) {
    double* vif = reinterpret_cast<double*>(scratch);
    unsigned long long* ngas = scratch + kNoallocMaxBubbles;
    int cb = -1;
    double cv = 0.0;
    unsigned long long cg = 0ull;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint8_t t = flags[i] & 15;
        if (!(t & (LBM_CELL_INTERFACE | LBM_CELL_GAS))) continue;
        const int b = owner[i];
        if (b < 0 || b >= nbub) continue;
        if (b != cb) {
            if (cb >= 0) {
                if (cv != 0.0) atomicAdd(&vif[cb], cv);
                if (cg) atomicAdd(&ngas[cb], cg);
            }
            cb = b;
            cv = 0.0;
            cg = 0ull;
        }
        if (t & LBM_CELL_INTERFACE) cv += 1.0 - (double)phi[i];
        else cg++;
    }
    if (cb >= 0) {
        if (cv != 0.0) atomicAdd(&vif[cb], cv);
        if (cg) atomicAdd(&ngas[cb], cg);
    }
}

__global__ void bubble_volumes_static_finish(int nbub, const unsigned long long* scratch, double* volumes) {
    const double* vif = reinterpret_cast<const double*>(scratch);
    const unsigned long long* ngas = scratch + kNoallocMaxBubbles;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbub; b += gridDim.x * blockDim.x)
        volumes[b] = (double)ngas[b] + vif[b];
}

// once per device, with it current: the device address of the static scratch, the device's
// multiprocessor count, and both kernels loaded (under CUDA's lazy module loading a kernel's
// code is loaded at its first use, which takes device memory: done here, at set-up)
int setup_current_device(DeviceSetup* out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return LBM_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& s = g_setup[dev];
    if (!s.scratch) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_bubble_scratch);
        if (e != cudaSuccess || !p) {
            std::fprintf(stderr, "lbm: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
            return LBM_ECUDA;
        }
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || sms < 1) {
            std::fprintf(stderr, "lbm: multiprocessor count query failed: %s\n", cudaGetErrorString(e));
            return LBM_ECUDA;
        }
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, bubble_volumes_static_kernel)) != cudaSuccess ||
            (e = cudaFuncGetAttributes(&fa, bubble_volumes_static_finish)) != cudaSuccess) {
            std::fprintf(stderr, "lbm: kernel load failed: %s\n", cudaGetErrorString(e));
            return LBM_ECUDA;
        }
        s.sms = sms;
        s.scratch = static_cast<unsigned long long*>(p);
    }
    *out = s;
    return LBM_OK;
}

int launch_error(cudaError_t e) {
    if (e == cudaSuccess) return LBM_OK;
    std::fprintf(stderr, "lbm_bubble_volumes_noalloc: launch failed: %s\n", cudaGetErrorString(e));
    return LBM_ECUDA;
}

}  // namespace

extern "C" int lbm_bubble_volumes_noalloc(const uint8_t* flags, const int32_t* owner, const float* phi,
                                          size_t n_cells, int n_bubbles, double* volumes, void* cuda_stream) {
    if (!flags || !owner || !phi || !volumes || n_cells == 0) return LBM_EINVAL;
    if (n_bubbles < 1 || n_bubbles > kNoallocMaxBubbles) {
        std::fprintf(stderr, "lbm_bubble_volumes_noalloc: %d bubbles, at most %d supported\n", n_bubbles,
                     kNoallocMaxBubbles);
        return LBM_EINVAL;
    }
    DeviceSetup dev;
    int rc = setup_current_device(&dev);
    if (rc) return rc;
    unsigned long long* scratch = dev.scratch;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the scratch keeps the previous call's sums: clear the part this call uses
    if (cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * n_bubbles, s) != cudaSuccess) return LBM_ECUDA;
    if (cudaMemsetAsync(scratch + kNoallocMaxBubbles, 0, sizeof(unsigned long long) * n_bubbles, s) != cudaSuccess)
        return LBM_ECUDA;
    size_t blocks = (n_cells + 255) / 256;
    if (blocks > (size_t)dev.sms * 8) blocks = (size_t)dev.sms * 8;   // grid-stride beyond 8 blocks per SM
    // each launch's own error (the return value), not an earlier one still pending on this thread
    {
        void* args[] = {(void*)&flags, (void*)&owner, (void*)&phi, (void*)&n_cells, (void*)&n_bubbles, (void*)&scratch};
        if ((rc = launch_error(cudaLaunchKernel((const void*)bubble_volumes_static_kernel, dim3((unsigned)blocks),
                                                dim3(256), args, 0, s))))
            return rc;
    }
    {
        const unsigned long long* cs = scratch;
        void* args[] = {(void*)&n_bubbles, (void*)&cs, (void*)&volumes};
        return launch_error(cudaLaunchKernel((const void*)bubble_volumes_static_finish, dim3((n_bubbles + 127) / 128),
                                             dim3(128), args, 0, s));
    }
}
