// hmi_cc.cu -- connected components across 32x32 blocks and the pointer
// (Mouse module, Sec. 2: the binary image's hand zone becomes a pointer with a
// position and a click state).
//   k_finish   one CTA per stream: union-find over the block components that
//              touch across block borders (8-connected), the root of every set
//              being its component with the smallest key (smallest pixel
//              index: the larger-key root is hooked under the smaller), the
//              statistics of non-roots added into their roots, the largest
//              root (ties: smaller label), the pointer and the click state
//   k_labels   per-pixel labels on demand (label = root key), same component
//              enumeration as the tick's block pass
// Every retry loop is bounded; overruns set an error flag in the stream state.
#include "hmi_ccfill.cuh"
#include "hmi_finish.cuh"
#include "hmi_internal.cuh"

namespace hmi {

constexpr int kActCap = 2048;
constexpr int kRecCap = 1024;
template <int NT>
using FinishSmemK = FinishSmem<NT, kActCap, kRecCap>;

// One CTA of NT threads per stream: the merge of its block components.
template <int NT>
__global__ void __launch_bounds__(NT) k_finish(BatchDev b)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FinishSmemK<NT> &S = *reinterpret_cast<FinishSmemK<NT> *>(smem_raw);
    if (threadIdx.x == 0 && blockIdx.x == 0) {   // k_skin and k_block_cc are done with their lists
        *b.cc_count = 0u;
        *b.skin_count = 0u;
    }
    const TickIO io = b.io[blockIdx.x];
    if (io.frame == nullptr) return;             // no frame this tick: pointer and click unchanged
    finish_stream<NT, kActCap, kRecCap>(b.ds[blockIdx.x], io, S, b.err,
                                        b.loop_limit ? b.loop_limit : kLoopLimit);
}

// Labels of one stream: warp per 32x32 block.
__global__ void __launch_bounds__(kThreads) k_labels(const DevStream *dsp, int32_t *labels)
{
    const DevStream &D = *dsp;
    const int lane = threadIdx.x & 31;
    const int blk = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nblk = D.bh * D.nwords;
    if (blk >= nblk) return;   // warp-uniform
    const int by = blk / D.nwords, bx = blk - by * D.nwords;
    const int y = by * kBlock + lane, xb = bx * kWordPx;
    const int npx = min(kWordPx, D.w - xb);
    const uint32_t *bits = D.bits_p[min(D.st->last_phase, 2u)];   // the last finished frame's mask
    uint32_t m = bits[(long long)y * D.nwords + bx];
    int32_t *row = labels + (long long)y * D.w + xb;
    if (y < D.h)
        for (int i = 0; i < npx; ++i) row[i] = -1;
    uint32_t *err = &D.st->err;
    int j = 0;
    while (__any_sync(kFull, m != 0u)) {
        int r0, c0;
        const uint32_t c = cc_extract_first(m, lane, &r0, &c0);
        m &= ~c;
        int32_t lab = -1;
        if (lane == 0 && j < kSlots) {
            const uint32_t root = find_root(D.parent, (uint32_t)blk * kSlots + (uint32_t)j, err);
            lab = (int32_t)D.comp[root].key;
        }
        lab = __shfl_sync(kFull, lab, 0);
        if (y < D.h)
            for (int i = 0; i < npx; ++i)
                if ((c >> i) & 1u) row[i] = lab;
        ++j;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int NT>
static cudaError_t launch_finish_nt(const BatchDev &b, cudaStream_t cs)
{
    static bool attr_set[64] = {};   // the shared-memory opt-in is per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(k_finish<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(FinishSmemK<NT>));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    k_finish<NT><<<b.n, NT, sizeof(FinishSmemK<NT>), cs>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_finish(const BatchDev &b, cudaStream_t cs)
{
    switch (b.merge_threads) {
    case 256: return launch_finish_nt<256>(b, cs);
    case 1024: return launch_finish_nt<1024>(b, cs);
    default: return launch_finish_nt<512>(b, cs);
    }
}

cudaError_t launch_labels(const DevStream *ds_dev, const DevStream &ds, int32_t *labels,
                          cudaStream_t cs)
{
    const long long nblk = (long long)ds.bh * ds.nwords;
    const unsigned grid = (unsigned)((nblk * 32 + kThreads - 1) / kThreads);
    k_labels<<<grid, kThreads, 0, cs>>>(ds_dev, labels);
    return cudaGetLastError();
}

}  // namespace hmi
