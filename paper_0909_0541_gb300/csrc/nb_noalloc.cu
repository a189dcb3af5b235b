// nb_noalloc.cu -- Morton order of a particle set without allocating: the
// root cube, 63-bit Morton keys and the stable radix sort that nb_build_tree
// runs first, with every scratch buffer taken from one file-scope device
// array instead of a context.
//
// Who needs this: code that may not call cudaMalloc.  cudaFree synchronises
// the whole device, which a caller in the middle of other streams' work may
// not allow, and in a process where another allocator (for example a deep-
// learning framework's caching allocator) has already reserved most of the
// device memory a raw cudaMalloc can fail.  Such callers hand in their
// inputs and outputs and get the sort order back with no allocation.
//
// The scratch array below lives in every GPU that loads libnb for as long as
// the process runs (NB_NOALLOC_SCRATCH_BYTES, about 12.9 MB).  Host code
// cannot use the array's name as a device address, so the first call on each
// device looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it for the life of the process; a cudaDeviceReset of
// that device invalidates the cached address, so the entry point must not be
// called again after one.  All calls share the array and it keeps the last
// call's contents: the error word is cleared at the start of each call and
// every other buffer is fully written before it is read.  Calls that overlap
// on the GPU (several host threads, or streams that run concurrently) race on
// the array.  Each call ends by synchronising its stream, to read the error
// word.
#include <mutex>

#include "nb_internal.cuh"

#define NA_MAX_N ((int64_t)NB_NOALLOC_MAX_N)
#define NA_TILES ((NA_MAX_N + NB_RS_TILE - 1) / NB_RS_TILE)
#define NA_HIST (256 * NA_TILES + 1)
#define NA_BSUM ((NA_HIST + 2047) / 2048 + 2)
#define NA_BBOX_BLOCKS 512

#define NA_ALIGN(x) ((((size_t)(x)) + 255) & ~(size_t)255)
#define NA_OFF_KEYS_ALT ((size_t)0)
#define NA_OFF_IDX_ALT NA_ALIGN(NA_OFF_KEYS_ALT + sizeof(uint64_t) * NA_MAX_N)
#define NA_OFF_HIST NA_ALIGN(NA_OFF_IDX_ALT + sizeof(uint32_t) * NA_MAX_N)
#define NA_OFF_BSUM NA_ALIGN(NA_OFF_HIST + sizeof(uint32_t) * NA_HIST)
#define NA_OFF_BBOX NA_ALIGN(NA_OFF_BSUM + sizeof(int32_t) * NA_BSUM)
#define NA_OFF_ROOT NA_ALIGN(NA_OFF_BBOX + sizeof(double) * 6 * NA_BBOX_BLOCKS)
#define NA_OFF_ERR NA_ALIGN(NA_OFF_ROOT + sizeof(double) * 8)
#define NB_NOALLOC_SCRATCH_BYTES NA_ALIGN(NA_OFF_ERR + sizeof(unsigned))

static __device__ __align__(256) unsigned char nb_noalloc_scratch[NB_NOALLOC_SCRATCH_BYTES];

#define NA_MAX_DEVICES 64
static void *g_scratch[NA_MAX_DEVICES];
static std::mutex g_scratch_mu;

// device address of the scratch array on the current device (set-up on the
// first call per device)
static int scratch_base(unsigned char **base)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return NB_ERR_CUDA;
    }
    if (dev < 0 || dev >= NA_MAX_DEVICES) return NB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, nb_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return NB_ERR_CUDA;
        }
        g_scratch[dev] = p;
    }
    *base = (unsigned char *)g_scratch[dev];
    return NB_OK;
}

extern "C" int nb_morton_order_noalloc(const double *pos_dev, int64_t n, uint64_t *keys_dev,
                                       int32_t *perm_dev, void *stream)
{
    if (n < 0 || n > NA_MAX_N || (n > 0 && (!pos_dev || !keys_dev || !perm_dev)))
        return NB_ERR_INVALID_ARG;
    if (n == 0) return NB_OK;
    unsigned char *base = nullptr;
    int rc = scratch_base(&base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t *keys_alt = (uint64_t *)(base + NA_OFF_KEYS_ALT);
    uint32_t *idx_alt = (uint32_t *)(base + NA_OFF_IDX_ALT);
    uint32_t *hist = (uint32_t *)(base + NA_OFF_HIST);
    int32_t *bsum = (int32_t *)(base + NA_OFF_BSUM);
    double *bbox = (double *)(base + NA_OFF_BBOX);
    double *root = (double *)(base + NA_OFF_ROOT);
    unsigned *err = (unsigned *)(base + NA_OFF_ERR);
    unsigned bits = 0;
    if (cudaMemsetAsync(err, 0, sizeof(unsigned), s) != cudaSuccess) goto cuda_fail;
    nb_launch_keys_raw(pos_dev, n, bbox, NA_BBOX_BLOCKS, root, keys_dev, (uint32_t *)perm_dev,
                       err, s);
    nb_radix_sort_raw(keys_dev, keys_alt, (uint32_t *)perm_dev, idx_alt, hist, bsum, n, s);
    if (cudaGetLastError() != cudaSuccess) goto cuda_fail;
    if (cudaMemcpyAsync(&bits, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        goto cuda_fail;
    return bits & NB_EF_NONFINITE ? NB_ERR_NONFINITE : NB_OK;
cuda_fail:
    cudaGetLastError();
    return NB_ERR_CUDA;
}
