// noalloc.cu — ||psi||^2 without any device allocation.
//
// Some callers cannot call cudaMalloc: their device memory is already entirely handed
// to their own allocator (a framework's caching pool at its limit), or they run a
// latency-critical loop in which an allocation's implicit device-wide synchronisation
// is not acceptable.  sv_norm_noalloc serves them: the caller passes the state and a
// device output, and the per-block partial sums go to a file-scope static device
// array of fixed size (every GPU that loads this library keeps it until exit).
#include <cuda_runtime.h>

#include <mutex>

#include "sv.h"

namespace svh {
sv_status set_error(sv_status s, const char* msg);
}

namespace {

constexpr int kChunkLog2 = 18;                      // amplitudes per partial sum
constexpr int kMaxPartials = 1 << 14;               // 128 KiB of FP64 partial sums
constexpr uint32_t kMaxQubits = kChunkLog2 + 14;     // 32

static __device__ __align__(256) double g_partials[kMaxPartials];

// Host-side stand-in for g_partials is not a device address: the real address is
// looked up once per device, with that device current.
std::mutex g_mu;
void* g_addr[64] = {};

template <typename C>
__global__ void __launch_bounds__(256) k_norm_chunks(const C* __restrict__ psi, uint64_t n_amp,
                                                     double* __restrict__ partials) {
    __shared__ double ws[8];
    const uint64_t lo = (uint64_t)blockIdx.x << kChunkLog2;
    const uint64_t hi = lo + (1ull << kChunkLog2) < n_amp ? lo + (1ull << kChunkLog2) : n_amp;
    double acc = 0.0;
    if (sizeof(C) == 8) {
        // FP32 partial sums over 16 complex64 amplitudes, FP64 above that
        const float4* p = reinterpret_cast<const float4*>(psi);
        uint64_t i = lo / 2 + threadIdx.x;
        for (; i + 7 * 256 < hi / 2; i += 8 * 256) {
            float s = 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float4 v = p[i + u * 256];
                s += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
            }
            acc += (double)s;
        }
        for (; i < hi / 2; i += 256) {
            const float4 v = p[i];
            acc += (double)(v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w);
        }
    } else {
        const double2* p = reinterpret_cast<const double2*>(psi);
        for (uint64_t i = lo + threadIdx.x; i < hi; i += 256) {
            const double2 v = p[i];
            acc += v.x * v.x + v.y * v.y;
        }
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += ws[w];
        partials[blockIdx.x] = s;   // every partial this call reads is written first
    }
}

// out = sum of partials[0..n), fixed order (strided sums, then a fixed tree)
__global__ void __launch_bounds__(256) k_sum_partials(const double* __restrict__ partials, uint32_t n,
                                                      double* __restrict__ out) {
    __shared__ double sm[256];
    double acc = 0.0;
    for (uint32_t i = threadIdx.x; i < n; i += 256) acc += partials[i];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

}  // namespace

extern "C" sv_status sv_norm_noalloc(const void* dev_state, uint32_t n_qubits, sv_dtype dtype,
                                     void* cuda_stream, double* dev_out) {
    if (!dev_state || !dev_out) return svh::set_error(SV_ERR_ARG, "null argument");
    if (dtype != SV_C64 && dtype != SV_C128) return svh::set_error(SV_ERR_ARG, "bad dtype");
    if (n_qubits < 1 || n_qubits > kMaxQubits)
        return svh::set_error(SV_ERR_ARG,
                              "n_qubits must be in [1, 32]: the static scratch holds 2^14 partial sums "
                              "of 2^18 amplitudes each");
    if ((uintptr_t)dev_state & 15) return svh::set_error(SV_ERR_ARG, "state must be 16-byte aligned");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return svh::set_error(SV_ERR_CUDA, "no current CUDA device");
    }
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            // first call on this device: the device is current, so this resolves the
            // device copy of the array (and loads the module if needed)
            cudaError_t e = cudaGetSymbolAddress(&g_addr[dev], g_partials);
            if (e != cudaSuccess) {
                g_addr[dev] = nullptr;
                return svh::set_error(SV_ERR_CUDA, cudaGetErrorString(e));
            }
        }
        scratch = g_addr[dev];
    }
    const uint64_t n_amp = 1ull << n_qubits;
    const uint32_t nblocks = (uint32_t)((n_amp + (1ull << kChunkLog2) - 1) >> kChunkLog2);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (dtype == SV_C64)
        k_norm_chunks<float2><<<nblocks, 256, 0, s>>>((const float2*)dev_state, n_amp, (double*)scratch);
    else
        k_norm_chunks<double2><<<nblocks, 256, 0, s>>>((const double2*)dev_state, n_amp, (double*)scratch);
    k_sum_partials<<<1, 256, 0, s>>>((const double*)scratch, nblocks, dev_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return svh::set_error(SV_ERR_CUDA, cudaGetErrorString(e));
    return SV_OK;
}
