// hmi_noalloc.cu -- brightness gain of one frame without any device allocation.
//
// Some callers cannot call cudaMalloc: code on a real-time path where an
// allocation may synchronise the device and stall the frame, or a host
// application that has handed all device memory to its own pool.  For them,
// hmi_frame_gain_noalloc computes the same Q16 brightness gain that the
// per-frame path derives from the frame's luma sum, using only a fixed scratch
// array compiled into this library (one per GPU that loads it, held until the
// process exits) and the buffers the caller passes in.
//
// Scratch: kNaCtas 64-bit partial sums (one per CTA) and one completion
// counter, 32 KiB + 256 B.  Each CTA covers exactly kNaChunksPerCta 16-pixel
// chunks, so the largest frame has kNaCtas * kNaChunksPerCta chunks
// (8192 x 8192 pixels); larger frames are rejected.  Every call uses the same
// array: calls that overlap on the GPU (on different streams, or from
// different threads) race and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "hmi_internal.cuh"

namespace hmi {
namespace {

constexpr int kNaCtas = 4096;
constexpr int kNaChunksPerCta = 1024;
constexpr int kNaCounter = kNaCtas;       // index of the completion counter
constexpr int kNaMaxDevices = 64;

// partial sums [0, kNaCtas) and the counter at kNaCounter
static __device__ __align__(256) unsigned long long g_na_scratch[kNaCtas + 32];

__device__ __forceinline__ uint32_t na_luma8(uint32_t r, uint32_t g, uint32_t b)
{
    return (77u * r + 150u * g + 29u * b + 128u) >> 8;
}

// One CTA per kNaChunksPerCta chunks of the (row, 16-px chunk) grid.  The last
// CTA to finish adds the partial sums and writes the clamped Q16 gain, then
// returns the counter to zero.
__global__ void __launch_bounds__(256)
k_frame_gain_noalloc(const uint8_t *__restrict__ frame, int w, int h, int vec, long long chunks,
                     unsigned long long syref, uint32_t gmin, uint32_t gmax, uint32_t *gain_out,
                     unsigned long long *scratch)
{
    __shared__ unsigned long long red[8];
    __shared__ bool is_last;
    const int cpr = (w + 15) / 16;
    const long long c0 = (long long)blockIdx.x * kNaChunksPerCta;
    const long long c1 = min(chunks, c0 + kNaChunksPerCta);
    unsigned long long acc = 0;
    for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        const int y = (int)(c / cpr), x0 = (int)(c - (long long)y * cpr) * 16;
        const int npx = min(16, w - x0);
        const uint8_t *p = frame + ((long long)y * w + x0) * 3;
        uint32_t sum = 0;
        if (vec) {
            const uint4 *q = reinterpret_cast<const uint4 *>(p);
            const uint4 a = __ldg(q), b = __ldg(q + 1), d = __ldg(q + 2);
            const uint32_t f[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, d.x, d.y, d.z, d.w};
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int o = 3 * k;
                const uint32_t r = (f[o >> 2] >> (8 * (o & 3))) & 0xffu;
                const uint32_t g = (f[(o + 1) >> 2] >> (8 * ((o + 1) & 3))) & 0xffu;
                const uint32_t bl = (f[(o + 2) >> 2] >> (8 * ((o + 2) & 3))) & 0xffu;
                sum += na_luma8(r, g, bl);
            }
        } else {
            for (int k = 0; k < npx; ++k) sum += na_luma8(p[3 * k], p[3 * k + 1], p[3 * k + 2]);
        }
        acc += sum;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        scratch[blockIdx.x] = t;
        __threadfence();
        is_last = atomicAdd(&scratch[kNaCounter], 1ull) == (unsigned long long)(gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    unsigned long long part = 0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x)
        part += *(volatile unsigned long long *)&scratch[i];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long sy = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) sy += red[i];
        unsigned long long g = (sy == 0) ? 65536ull : ((syref << 16) + sy / 2) / sy;
        if (g < gmin) g = gmin;
        if (g > gmax) g = gmax;
        *gain_out = (uint32_t)g;
        scratch[kNaCounter] = 0;
    }
}

std::mutex g_na_mu;
void *g_na_ptr[kNaMaxDevices] = {};

// Device address of the scratch array on device `dev` (current).  Outside a
// stream capture it is looked up on every call, so that a device reset or a
// new primary context never leaves a stale address behind; inside a capture
// the address found by the last call outside one is used (none yet: an error,
// since the lookup may have to load the module, which a capture forbids).
cudaError_t na_scratch(int dev, cudaStream_t cs, unsigned long long **out)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(cs, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = p;
    } else if (!g_na_ptr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = static_cast<unsigned long long *>(g_na_ptr[dev]);
    return cudaSuccess;
}

// Memory that a kernel on device `dev` may read (device_only false: device or
// managed memory of that device, or pinned / registered host memory mapped at
// the same address) or write (device_only true: device or managed memory of
// that device only).
bool na_reachable(const void *p, int dev, bool device_only)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeDevice) return at.device == dev;
    if (at.type == cudaMemoryTypeManaged) return true;
    return !device_only && at.type == cudaMemoryTypeHost && at.devicePointer == p;
}

}  // namespace
}  // namespace hmi

extern "C" int hmi_frame_gain_noalloc(const uint8_t *frame, int w, int h, uint64_t syref,
                                      uint32_t gain_min_q16, uint32_t gain_max_q16,
                                      uint32_t *gain_out, void *cuda_stream)
{
    using namespace hmi;
    if (!frame || !gain_out || w < 1 || h < 1 || w > kMaxDim || h > kMaxDim ||
        gain_min_q16 > gain_max_q16 || gain_max_q16 > (1u << 24) ||
        (reinterpret_cast<uintptr_t>(gain_out) & 3u) != 0 ||
        syref > 255ull * (uint64_t)w * (uint64_t)h)   // no frame of this size has a larger luma sum
        return set_error(HMI_ERR_INVALID_ARG);
    const long long chunks = (long long)h * ((w + 15) / 16);
    if (chunks > (long long)kNaCtas * kNaChunksPerCta) return set_error(HMI_ERR_INVALID_ARG);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
        (void)cudaGetLastError();
        return set_error(HMI_ERR_DEVICE);
    }
    // the frame must be readable and the gain writable by this device's kernels
    if (!na_reachable(frame, dev, false) || !na_reachable(gain_out, dev, true))
        return set_error(HMI_ERR_INVALID_ARG);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(cuda_stream);
    unsigned long long *scratch = nullptr;
    if (na_scratch(dev, cs, &scratch) != cudaSuccess) {
        (void)cudaGetLastError();
        return set_error(HMI_ERR_DEVICE);
    }
    // the completion counter must start at zero even if an earlier call was cut short
    if (cudaMemsetAsync(scratch + kNaCounter, 0, sizeof(unsigned long long), cs) != cudaSuccess) {
        (void)cudaGetLastError();
        return set_error(HMI_ERR_DEVICE);
    }
    const int vec = ((w % 16) == 0 && (reinterpret_cast<uintptr_t>(frame) & 15u) == 0) ? 1 : 0;
    const unsigned grid = (unsigned)((chunks + kNaChunksPerCta - 1) / kNaChunksPerCta);
    k_frame_gain_noalloc<<<grid, 256, 0, cs>>>(frame, w, h, vec, chunks, syref, gain_min_q16,
                                               gain_max_q16, gain_out, scratch);
    if (cudaGetLastError() != cudaSuccess) return set_error(HMI_ERR_DEVICE);
    return HMI_OK;
}
