// Cell binning (the (cell, id) particle sort) for callers that cannot
// allocate device memory.
//
// Some callers must not allocate GPU memory while they run: code that is
// being recorded into a CUDA graph (cudaMalloc is not a stream operation and
// cannot be captured), real-time loops where cudaMalloc/cudaFree would
// introduce an implicit device synchronisation, and hosts that own a fixed
// device-memory budget and hand libraries only the buffers they asked for.
// lbdps_bin_sort_noalloc serves them: the caller passes the positions and the
// two output buffers, and every temporary this sort needs lives in one
// file-scope device array of fixed size that is created when the library is
// loaded on a GPU and kept until the process exits.
#include "lbdps.h"
#include "lbdps_internal.cuh"

#include <cstdio>
#include <mutex>

namespace lbdpsk {
void set_last_error(const char *msg);
}

namespace {

constexpr int kMaxCells = 1 << 20;       // lattice cells per call
constexpr int kMaxParticles = 1 << 20;   // particles per call
constexpr int kScanTile = 4096;          // cells per block of the shared scan kernels
constexpr int kMaxBlockSums = kMaxCells / kScanTile + 2;
// radix sort of the cell keys: 8-bit digits, tiles of 256 particles (one per
// thread), a digit-major histogram of 256 bins x tiles
constexpr int kRadixBits = 8;
constexpr int kBins = 1 << kRadixBits;
constexpr int kRadixTile = 256;
constexpr int kRadixWarps = kRadixTile / 32;
constexpr int kMaxTiles = kMaxParticles / kRadixTile;
constexpr int kMaxHist = kBins * kMaxTiles;
static_assert(kMaxHist == kMaxCells, "the count array doubles as the scanned histogram");
static_assert(kRadixTile == kBins, "one thread per bin in the tile histogram");
constexpr size_t kScratchInts = (size_t)kMaxCells + 1           // counts, then digit offsets
                                + (size_t)kMaxHist               // digit histogram
                                + 5 * (size_t)kMaxParticles      // keys; keys and ids x 2
                                + (size_t)kMaxBlockSums;
constexpr int kMaxDevices = 64;

}  // namespace

// counts | digit histogram | keys | keys A | ids A | keys B | ids B | block sums
static __device__ __align__(256) int g_bin_scratch[kScratchInts];

namespace {

std::mutex g_setup_mutex;
int *g_scratch_ptr[kMaxDevices] = {};

// Cell key of each particle and the per-cell counts.  Each coordinate is
// clamped in FP64 before any conversion: below 0 (or NaN) to the first cell,
// at or above n[a] to the last, so the integer cast only sees [0, n[a]).
__global__ void k_na_keys(int dim, int n0, int n1, int n2, const double *P0, const double *P1,
                          const double *P2, int np, int *key, int *counts)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const int n[3] = {n0, n1, n2};
    const double *P[3] = {P0, P1, P2};
    int q[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        const double x = P[a][k];
        int v = 0;
        if (x >= 0.0) v = x < (double)n[a] ? (int)x : n[a] - 1;
        q[a] = v;
    }
    const int c = q[0] + n0 * (q[1] + n1 * q[2]);
    key[k] = c;
    atomicAdd(&counts[c], 1);
}

// Per-warp counts of each digit among the tile's particles, in shared
// memory: cnt[w][d] = particles of warp w with digit d.  Returns the
// particle's digit (kBins for a slot past the end) and the lanes of its warp
// holding the same digit.
__device__ __forceinline__ int tile_digit_counts(const int *keys, int np, int shift,
                                                 int (*cnt)[kBins], unsigned *peers)
{
    const int t = threadIdx.x, warp = t >> 5;
    const int item = blockIdx.x * kRadixTile + t;
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) cnt[w][t] = 0;
    __syncthreads();
    const int d = item < np ? (keys[item] >> shift) & (kBins - 1) : kBins;
    const unsigned same = __match_any_sync(0xffffffffu, d);
    if (d < kBins && (t & 31) == __ffs(same) - 1) cnt[warp][d] = __popc(same);
    __syncthreads();
    *peers = same;
    return d;
}

// hist[d * tiles + tile] = particles of the tile whose key has digit d
__global__ void __launch_bounds__(kRadixTile)
k_na_digit_hist(const int *keys, int np, int shift, int tiles, int *hist)
{
    __shared__ int cnt[kRadixWarps][kBins];
    unsigned peers;
    tile_digit_counts(keys, np, shift, cnt, &peers);
    int sum = 0;
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) sum += cnt[w][threadIdx.x];
    hist[threadIdx.x * tiles + blockIdx.x] = sum;
}

// Stable placement by digit: a particle goes to the scanned offset of (its
// digit, its tile) plus the number of particles before it in the tile with
// the same digit.  ids_in null: the id is the particle's index (first pass);
// keys_out null: only ids are written (last pass).
__global__ void __launch_bounds__(kRadixTile)
k_na_digit_scatter(const int *keys, const int *ids_in, int np, int shift, int tiles,
                   const int *offs, int *keys_out, int *ids_out)
{
    __shared__ int cnt[kRadixWarps][kBins];
    unsigned peers;
    const int d = tile_digit_counts(keys, np, shift, cnt, &peers);
    if (d >= kBins) return;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int item = blockIdx.x * kRadixTile + t;
    int rank = __popc(peers & ((1u << lane) - 1u));
    for (int w = 0; w < warp; ++w) rank += cnt[w][d];
    const int pos = offs[d * tiles + blockIdx.x] + rank;
    if (keys_out) keys_out[pos] = keys[item];
    ids_out[pos] = ids_in ? ids_in[item] : item;
}

int na_fail(int code, const char *msg)
{
    lbdpsk::set_last_error(msg);
    return code;
}

}  // namespace

extern "C" int lbdps_bin_sort_noalloc(int dim, const int n[3], int64_t np, const double *const pos[3],
                                      int *cell_start, int *order, void *stream)
{
    if ((dim != 2 && dim != 3) || !n || !pos || !cell_start || np < 0 || (np > 0 && !order))
        return na_fail(LBDPS_ERR_INVALID, "lbdps_bin_sort_noalloc: bad arguments");
    long long ncell = 1;
    int nn[3] = {1, 1, 1};
    for (int a = 0; a < dim; ++a) {
        if (n[a] < 1) return na_fail(LBDPS_ERR_INVALID, "lbdps_bin_sort_noalloc: n[a] must be positive");
        if (np > 0 && !pos[a]) return na_fail(LBDPS_ERR_INVALID, "lbdps_bin_sort_noalloc: NULL position array");
        nn[a] = n[a];
        ncell *= n[a];
        if (ncell > kMaxCells) break;
    }
    if (ncell > kMaxCells || np > kMaxParticles) {
        char buf[200];
        snprintf(buf, sizeof(buf),
                 "lbdps_bin_sort_noalloc: %lld%s cells / %lld particles exceed the fixed scratch "
                 "(at most %d cells and %d particles)",
                 ncell, ncell > kMaxCells ? "+" : "", (long long)np, kMaxCells, kMaxParticles);
        return na_fail(LBDPS_ERR_CAPACITY, buf);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return na_fail(LBDPS_ERR_CUDA, "lbdps_bin_sort_noalloc: no current CUDA device");
    }
    int *base = nullptr;
    {
        // one-time set-up per device, with that device current: the device
        // address of the scratch array (the host-side symbol is only a stand-in)
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_bin_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                char buf[160];
                snprintf(buf, sizeof(buf), "lbdps_bin_sort_noalloc: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(e));
                return na_fail(LBDPS_ERR_CUDA, buf);
            }
            g_scratch_ptr[dev] = (int *)p;
        }
        base = g_scratch_ptr[dev];
    }
    int *counts = base;                          // kMaxCells + 1; digit offsets later
    int *hist = counts + kMaxCells + 1;          // kMaxHist
    int *keys = hist + kMaxHist;                 // kMaxParticles each below
    int *keys_a = keys + kMaxParticles;
    int *ids_a = keys_a + kMaxParticles;
    int *keys_b = ids_a + kMaxParticles;
    int *ids_b = keys_b + kMaxParticles;
    int *block_sums = ids_b + kMaxParticles;     // kMaxBlockSums
    cudaStream_t st = (cudaStream_t)stream;
    const int npi = (int)np;
    const int nc = (int)ncell;
    const int tiles = (npi + kRadixTile - 1) / kRadixTile;
    if (lbdpsk::scan_block_count(nc) + 1 > kMaxBlockSums ||
        lbdpsk::scan_block_count(kBins * tiles) + 1 > kMaxBlockSums)
        return na_fail(LBDPS_ERR_CAPACITY, "lbdps_bin_sort_noalloc: scan scratch too small");

    // the counts must start at zero; the array keeps whatever the last call left
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)nc, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return na_fail(LBDPS_ERR_CUDA, "lbdps_bin_sort_noalloc: clearing the counts failed");
    }
    if (npi > 0) {
        k_na_keys<<<(npi + 255) / 256, 256, 0, st>>>(dim, nn[0], nn[1], nn[2], pos[0], pos[1],
                                                     dim > 2 ? pos[2] : nullptr, npi, keys, counts);
    }
    lbdpsk::launch_scan(counts, cell_start, block_sums, nc, st);
    if (npi > 0) {
        // (cell, id) order: least-significant-digit radix sort of the keys,
        // stable in every pass, starting from id order; as many 8-bit digits
        // as the largest key needs
        int passes = 1;
        while (passes < 3 && (long long)nc > (1ll << (kRadixBits * passes))) ++passes;
        const int nh = kBins * tiles;
        const int *kin = keys, *iin = nullptr;
        int *kout[2] = {keys_b, keys_a}, *iout[2] = {ids_b, ids_a};
        for (int pass = 0; pass < passes; ++pass) {
            const int shift = kRadixBits * pass;
            const bool last = pass == passes - 1;
            k_na_digit_hist<<<tiles, kRadixTile, 0, st>>>(kin, npi, shift, tiles, hist);
            lbdpsk::launch_scan(hist, counts, block_sums, nh, st);   // digit offsets
            int *ko = last ? nullptr : kout[pass & 1];
            int *io = last ? order : iout[pass & 1];
            k_na_digit_scatter<<<tiles, kRadixTile, 0, st>>>(kin, iin, npi, shift, tiles, counts,
                                                               ko, io);
            kin = ko;
            iin = io;
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        char buf[160];
        snprintf(buf, sizeof(buf), "lbdps_bin_sort_noalloc: launch failed: %s", cudaGetErrorString(e));
        return na_fail(LBDPS_ERR_CUDA, buf);
    }
    return LBDPS_OK;
}
