// lbm_noalloc.cu -- bubble volumes without any device allocation.
//
// Some callers cannot call cudaMalloc: code running where allocation is forbidden or
// deferred (inside an allocator hook, a signal-safe or real-time section, a host callback),
// or a host program whose memory budget is fixed and fully handed out before it starts.
// lbm_bubble_volumes_noalloc serves them: it is a variant of the bubble-volume reduction of
// lbm_step whose scratch (per-bubble partial sums) is a file-scope static device array, so
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
unsigned long long* g_scratch_addr[kNoallocMaxDevices] = {nullptr};

// Same sums as the step's bubble model: V_b = #gas cells of b + sum over interface cells of b
// of (1 - phi), FP64, from canonical inputs (types LBM_CELL_*, owner -1 for none).
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

// device address of the static scratch for the current device, looked up once per device
int scratch_for_current_device(unsigned long long** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return LBM_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_bubble_scratch);
        if (e != cudaSuccess || !p) {
            std::fprintf(stderr, "lbm: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
            return LBM_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_scratch_addr[dev];
    return LBM_OK;
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
    unsigned long long* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the scratch keeps the previous call's sums: clear the part this call uses
    if (cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * n_bubbles, s) != cudaSuccess) return LBM_ECUDA;
    if (cudaMemsetAsync(scratch + kNoallocMaxBubbles, 0, sizeof(unsigned long long) * n_bubbles, s) != cudaSuccess)
        return LBM_ECUDA;
    size_t blocks = (n_cells + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    bubble_volumes_static_kernel<<<(unsigned)blocks, 256, 0, s>>>(flags, owner, phi, n_cells, n_bubbles, scratch);
    bubble_volumes_static_finish<<<(n_bubbles + 127) / 128, 128, 0, s>>>(n_bubbles, scratch, volumes);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
