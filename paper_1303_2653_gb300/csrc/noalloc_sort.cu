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

#include <cmath>
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
constexpr size_t kScratchInts =
    (size_t)kMaxCells + 2 * (size_t)kMaxParticles + (size_t)kMaxBlockSums;
constexpr int kMaxDevices = 64;

}  // namespace

// counts[kMaxCells] | keys[kMaxParticles] | slots[kMaxParticles] | block sums
static __device__ __align__(256) int g_bin_scratch[kScratchInts];

namespace {

std::mutex g_setup_mutex;
int *g_scratch_ptr[kMaxDevices] = {};

__global__ void k_na_keys(int dim, int n0, int n1, int n2, const double *P0, const double *P1,
                          const double *P2, int np, int *key, int *counts)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const int n[3] = {n0, n1, n2};
    const double *P[3] = {P0, P1, P2};
    int q[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        int v = (int)floor(P[a][k]);
        v = v < 0 ? 0 : (v >= n[a] ? n[a] - 1 : v);
        q[a] = v;
    }
    const int c = q[0] + n0 * (q[1] + n1 * q[2]);
    key[k] = c;
    atomicAdd(&counts[c], 1);
}

__global__ void k_na_scatter(const int *key, int *counts, const int *cell_start, int *slots, int np)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const int c = key[k];
    const int old = atomicSub(&counts[c], 1);
    slots[cell_start[c] + old - 1] = k;
}

// Within a cell the particles are ordered by index (the particle id).
__global__ void k_na_rank(const int *key, const int *cell_start, const int *slots, int *order,
                          int np)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= np) return;
    const int k = slots[s];
    const int c = key[k];
    const int lo = cell_start[c], hi = cell_start[c + 1];
    int rank = 0;
    for (int q = lo; q < hi; ++q) rank += (slots[q] < k) ? 1 : 0;
    order[lo + rank] = k;
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
    if ((dim != 2 && dim != 3) || !n || !pos || !cell_start || (np > 0 && !order))
        return na_fail(LBDPS_ERR_INVALID, "lbdps_bin_sort_noalloc: bad arguments");
    long long ncell = 1;
    int nn[3] = {1, 1, 1};
    for (int a = 0; a < dim; ++a) {
        if (n[a] < 1) return na_fail(LBDPS_ERR_INVALID, "lbdps_bin_sort_noalloc: n[a] must be positive");
        if (np > 0 && !pos[a]) return na_fail(LBDPS_ERR_INVALID, "lbdps_bin_sort_noalloc: NULL position array");
        nn[a] = n[a];
        ncell *= n[a];
    }
    if (ncell > kMaxCells || np < 0 || np > kMaxParticles) {
        char buf[200];
        snprintf(buf, sizeof(buf),
                 "lbdps_bin_sort_noalloc: %lld cells / %lld particles exceed the fixed scratch "
                 "(at most %d cells and %d particles)",
                 ncell, (long long)np, kMaxCells, kMaxParticles);
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
    int *counts = base;
    int *keys = counts + kMaxCells;
    int *slots = keys + kMaxParticles;
    int *block_sums = slots + kMaxParticles;
    cudaStream_t st = (cudaStream_t)stream;
    const int npi = (int)np;
    const int nc = (int)ncell;
    if (lbdpsk::scan_block_count(nc) + 1 > kMaxBlockSums)
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
        k_na_scatter<<<(npi + 255) / 256, 256, 0, st>>>(keys, counts, cell_start, slots, npi);
        k_na_rank<<<(npi + 255) / 256, 256, 0, st>>>(keys, cell_start, slots, order, npi);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        char buf[160];
        snprintf(buf, sizeof(buf), "lbdps_bin_sort_noalloc: launch failed: %s", cudaGetErrorString(e));
        return na_fail(LBDPS_ERR_CUDA, buf);
    }
    return LBDPS_OK;
}
