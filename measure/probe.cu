// probe.cu -- gather-rate probe: the memory ceilings a record walk can reach on this device.
//
// The walk's hot loop is one dependent 32-byte record gather per edge crossing (Alg. "Parallel
// Geodesic Tracing CUDA Kernel": each thread reads the next face's data before it can choose
// the exit edge).  With the records of a mesh resident in L2, its ceiling is not the HBM copy
// bandwidth but the L2's, and with one gather in flight per thread, the rate at which chains of
// dependent gathers complete.  The three modes below measure:
//
//   SG_PROBE_STREAM    coalesced 16-byte loads sweeping the table (L2 read bandwidth once the
//                      table is L2-resident and larger than the L1s)
//   SG_PROBE_RANDOM    independent 32-byte record gathers at random positions (four per thread
//                      in flight): the L2 sector-gather rate
//   SG_PROBE_CHAIN     dependent chains: each record holds the index of the next one, a single
//                      random cycle through the table, and each thread follows it with one
//                      gather in flight, like a walker
//
// Records are 32 bytes, loaded through the read-only path either as the walk loads them (two
// 16-byte loads) or, with SG_PROBE_LD256, as one 256-bit load (sm_100 and later), which the
// L1 serves as one request instead of two.
//
// sg_probe_reduce measures the rate of random floating-point reductions into an accumulator table
// of the size of a mesh's gradient accumulator, the other traffic of the backward re-walk:
//
//   SG_PROBE_RED8      8-byte reductions (two floats) into L2
//   SG_PROBE_RED16     16-byte reductions (four floats) into L2
//   SG_PROBE_RED_DSM   the table spread over the shared memory of a thread-block cluster (one CTA
//                      of 896 threads per SM), each reduction two 4-byte red.shared::cluster on
//                      the owning CTA, the table flushed to global memory at the end
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

// Measurement-only library (libsgeo_probe.so), built beside the exponential-map library and
// loaded by the benchmark; it is not part of the exponential map's C ABI.  Return codes: 0 ok,
// 1 invalid argument, 4 CUDA error, 5 out of device memory.
#define SG_PROBE_STREAM 0
#define SG_PROBE_RANDOM 1
#define SG_PROBE_CHAIN 2
#define SG_PROBE_LD256 4
#define SG_PROBE_RED8 0
#define SG_PROBE_RED16 1
#define SG_PROBE_RED_DSM 2
typedef int sg_probe_status;
#define SG_OK 0
#define SG_ERR_INVALID_ARG 1
#define SG_ERR_CUDA 4
#define SG_ERR_OOM 5

namespace {

template <bool W>
__device__ __forceinline__ void ld_rec(const int4 *__restrict__ p, int4 &a, int4 &b) {
    if (W) {
        asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
            : "l"(p));
    } else {
        a = __ldg(p);
        b = __ldg(p + 1);
    }
}

__global__ void __launch_bounds__(1024) k_probe_stream(const int4 *__restrict__ t, int64_t n16, int32_t passes,
                                                       unsigned *sink) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    unsigned acc = 0;
    for (int32_t p = 0; p < passes; ++p)
        for (int64_t i = tid; i < n16; i += nth) {
            const int4 a = __ldg(t + i);
            acc ^= (unsigned)(a.x ^ a.y ^ a.z ^ a.w);
        }
    if (acc == 0x9e3779b9u) sink[0] = acc;  // never true for the table's contents; keeps the loads
}

// records indexed with a mask: the table holds a power-of-two count of records
template <bool W>
__global__ void __launch_bounds__(1024) k_probe_random(const int4 *__restrict__ t, uint32_t mask, int32_t loads,
                                                       unsigned *sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x = tid * 2654435761u + 12345u;
    unsigned acc = 0;
    for (int32_t k = 0; k < loads; k += 4) {
        uint32_t r[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            x = x * 1664525u + 1013904223u;   // LCG step (Numerical Recipes constants)
            r[j] = (x >> 7) & mask;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int4 a, b;
            ld_rec<W>(t + 2 * (size_t)r[j], a, b);
            acc ^= (unsigned)(a.x ^ a.w ^ b.y ^ b.z);
        }
    }
    if (acc == 0x9e3779b9u) sink[0] = acc;
}

template <bool W>
__global__ void __launch_bounds__(1024) k_probe_chain(const int4 *__restrict__ t, uint32_t nrec, int32_t loads,
                                                      unsigned *sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t idx = (uint32_t)(((uint64_t)tid * 2654435761u) % nrec);
    unsigned acc = 0;
    for (int32_t k = 0; k < loads; ++k) {
        int4 a, b;
        ld_rec<W>(t + 2 * (size_t)idx, a, b);
        acc ^= (unsigned)(a.w ^ b.x ^ b.w);
        idx = (uint32_t)a.x;                  // in [0, nrec): written by the host below
    }
    if (acc == 0x9e3779b9u) sink[0] = acc ^ idx;
}

// an index in [0, n) from a linear congruential step (Numerical Recipes constants)
__device__ __forceinline__ uint32_t next_index(uint32_t &x, uint32_t n) {
    x = x * 1664525u + 1013904223u;
    return (uint32_t)(((uint64_t)(x >> 8) * n) >> 24);
}

__global__ void __launch_bounds__(256) k_probe_red8(float2 *acc, uint32_t n, int32_t iters) {
    uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
    for (int32_t i = 0; i < iters; ++i) atomicAdd(acc + next_index(x, n), make_float2(1.f, 2.f));
}

__global__ void __launch_bounds__(256) k_probe_red16(float4 *acc, uint32_t n, int32_t iters) {
    uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
    for (int32_t i = 0; i < iters; ++i) atomicAdd(acc + next_index(x, n), make_float4(1.f, 2.f, 3.f, 4.f));
}

// entries [r slice, (r+1) slice) of the n-entry float2 table live in the shared memory of the
// cluster's CTA r; magic = floor(2^32 / slice) gives r = e / slice with one correction
__global__ void __launch_bounds__(896, 1) k_probe_red_dsm(float2 *acc, uint32_t n, uint32_t slice, uint32_t magic,
                                                          int32_t iters) {
    extern __shared__ float2 part[];
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    for (uint32_t i = threadIdx.x; i < slice; i += blockDim.x) part[i] = make_float2(0.f, 0.f);
    cl.sync();  // every CTA of the cluster has zeroed its part before any remote reduction
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(part);
    uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
    for (int32_t i = 0; i < iters; ++i) {
        const uint32_t e = next_index(x, n);
        uint32_t r = __umulhi(e, magic);
        if (e - r * slice >= slice) ++r;  // r = e / slice < cluster size, since n <= cluster * slice
        const uint32_t local = base + 8u * (e - r * slice);
        asm volatile(
            "{\n\t.reg .b32 ra;\n\tmapa.shared::cluster.u32 ra, %0, %1;\n\t"
            "red.shared::cluster.add.f32 [ra], %2;\n\tred.shared::cluster.add.f32 [ra+4], %3;\n\t}" ::"r"(local),
            "r"(r), "f"(1.f), "f"(2.f)
            : "memory");
    }
    cl.sync();  // no CTA leaves while others may still reduce into its part
    const uint32_t e0 = cl.block_rank() * slice;
    for (uint32_t i = threadIdx.x; i < slice && e0 + i < n; i += blockDim.x) {
        const float2 c = part[i];
        if (c.x != 0.f || c.y != 0.f) atomicAdd(acc + e0 + i, c);
    }
}

uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" sg_probe_status sg_probe_gather(int32_t mode, int64_t table_bytes, int32_t blocks_per_sm, int32_t threads,
                                     int32_t loads, double *out_seconds, double *out_bytes) {
    if (!out_seconds || !out_bytes) return SG_ERR_INVALID_ARG;
    const bool w256 = (mode & SG_PROBE_LD256) != 0;
    mode &= ~SG_PROBE_LD256;
    if (mode < SG_PROBE_STREAM || mode > SG_PROBE_CHAIN) return SG_ERR_INVALID_ARG;
    if (table_bytes < 4096 || table_bytes > ((int64_t)1 << 31)) return SG_ERR_INVALID_ARG;
    if (blocks_per_sm < 1 || blocks_per_sm > 32 || threads < 32 || threads > 1024 || (threads & 31)) return SG_ERR_INVALID_ARG;
    if (loads < 4 || loads > (1 << 20)) return SG_ERR_INVALID_ARG;
    // a power-of-two count of 32-byte records, at most table_bytes
    uint32_t nrec = 1;
    while ((int64_t)nrec * 2 * 32 <= table_bytes && nrec < (1u << 29)) nrec *= 2;
    const size_t bytes = (size_t)nrec * 32;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SG_ERR_CUDA;
    // records: {next, i, ~i, i ^ salt}, {salt, i * 3, i + 7, next ^ i}; next is a single cycle
    // through every record (Sattolo's shuffle), so each chain visits distinct records
    std::vector<int32_t> h((size_t)nrec * 8);
    std::vector<uint32_t> perm(nrec);
    for (uint32_t i = 0; i < nrec; ++i) perm[i] = i;
    uint64_t seed = 0x5eed0fa11ULL;
    for (uint32_t i = nrec - 1; i > 0; --i) {
        const uint32_t j = (uint32_t)(splitmix64(seed) % i);  // j < i: one cycle
        const uint32_t tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
    }
    for (uint32_t i = 0; i < nrec; ++i) {
        int32_t *r = h.data() + 8 * (size_t)i;
        const int32_t salt = (int32_t)(splitmix64(seed) & 0x7fffffff);
        r[0] = (int32_t)perm[i]; r[1] = (int32_t)i; r[2] = ~(int32_t)i; r[3] = (int32_t)i ^ salt;
        r[4] = salt; r[5] = (int32_t)(i * 3u); r[6] = (int32_t)(i + 7u); r[7] = (int32_t)(perm[i] ^ i);
    }
    int4 *t = nullptr;
    unsigned *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sg_probe_status st = SG_OK;
    if (cudaMalloc((void **)&t, bytes) != cudaSuccess || cudaMalloc((void **)&sink, 64) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(t);
        return SG_ERR_OOM;
    }
    const unsigned grid = (unsigned)sms * (unsigned)blocks_per_sm;
    const uint64_t nthreads = (uint64_t)grid * (uint64_t)threads;
    double moved = 0.0;
    float ms = 0.f;
    if (cudaMemcpy(t, h.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        st = SG_ERR_CUDA;
    } else {
        // one untimed launch brings the table into L2, then one timed launch
        for (int rep = 0; rep < 2; ++rep) {
            if (rep == 1) cudaEventRecord(e0, 0);
            if (mode == SG_PROBE_STREAM) {
                k_probe_stream<<<grid, threads>>>(t, (int64_t)(bytes / 16), loads, sink);
                moved = (double)bytes * loads;
            } else if (mode == SG_PROBE_RANDOM) {
                if (w256) k_probe_random<true><<<grid, threads>>>(t, nrec - 1, loads, sink);
                else k_probe_random<false><<<grid, threads>>>(t, nrec - 1, loads, sink);
                moved = 32.0 * (double)nthreads * (double)((loads + 3) / 4 * 4);
            } else {
                if (w256) k_probe_chain<true><<<grid, threads>>>(t, nrec, loads, sink);
                else k_probe_chain<false><<<grid, threads>>>(t, nrec, loads, sink);
                moved = 32.0 * (double)nthreads * (double)loads;
            }
            if (rep == 1) cudaEventRecord(e1, 0);
        }
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = SG_ERR_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(t);
    if (st == SG_OK && cudaGetLastError() != cudaSuccess) st = SG_ERR_CUDA;
    *out_seconds = st == SG_OK ? ms * 1e-3 : 0.0;
    *out_bytes = st == SG_OK ? moved : 0.0;
    return st;
}

// Random reductions into an accumulator table of table_bytes: `iters` per thread, one untimed and
// one timed launch.  SG_PROBE_RED8 / RED16: 8 blocks of 256 threads per SM.  SG_PROBE_RED_DSM: one
// CTA of 896 threads per SM in clusters of `cluster` CTAs (2..16), as many clusters as fit at once;
// SG_ERR_INVALID_ARG when the table's share per CTA exceeds the shared memory a block may use or
// no cluster of that size fits.  out_ops = reductions performed (of 8 or 16 bytes).
extern "C" sg_probe_status sg_probe_reduce(int32_t mode, int64_t table_bytes, int32_t cluster, int32_t iters,
                                           double *out_seconds, double *out_ops) {
    if (!out_seconds || !out_ops) return SG_ERR_INVALID_ARG;
    if (mode < SG_PROBE_RED8 || mode > SG_PROBE_RED_DSM) return SG_ERR_INVALID_ARG;
    if (table_bytes < 4096 || table_bytes > ((int64_t)1 << 28) || iters < 1 || iters > (1 << 16)) return SG_ERR_INVALID_ARG;
    if (mode == SG_PROBE_RED_DSM && (cluster < 2 || cluster > 16)) return SG_ERR_INVALID_ARG;
    int dev = 0, sms = 0, maxopt = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return SG_ERR_CUDA;
    const uint32_t n = (uint32_t)(table_bytes / (mode == SG_PROBE_RED16 ? 16 : 8));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    uint32_t slice = 0, magic = 0;
    int nclusters = 0;
    if (mode == SG_PROBE_RED_DSM) {
        slice = (n + (uint32_t)cluster - 1) / (uint32_t)cluster;
        const size_t smem = (size_t)slice * sizeof(float2);
        if (smem > (size_t)maxopt) return SG_ERR_INVALID_ARG;
        if (cudaFuncSetAttribute(k_probe_red_dsm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
            cudaFuncSetAttribute(k_probe_red_dsm, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
            cudaGetLastError();
            return SG_ERR_CUDA;
        }
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.blockDim = dim3(896);
        cfg.gridDim = dim3((unsigned)cluster);
        cfg.dynamicSmemBytes = smem;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_probe_red_dsm, &cfg) != cudaSuccess) {
            cudaGetLastError();
            return SG_ERR_CUDA;
        }
        if (nclusters < 1) return SG_ERR_INVALID_ARG;
        cfg.gridDim = dim3((unsigned)(nclusters * cluster));
        magic = (uint32_t)(0x100000000ull / slice);
    }
    void *acc = nullptr;
    if (cudaMalloc(&acc, (size_t)table_bytes) != cudaSuccess) {
        cudaGetLastError();
        return SG_ERR_OOM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sg_probe_status st = SG_OK;
    float ms = 0.f;
    double ops = 0.0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = SG_ERR_CUDA;
    for (int rep = 0; rep < 2 && st == SG_OK; ++rep) {
        if (cudaMemset(acc, 0, (size_t)table_bytes) != cudaSuccess) { st = SG_ERR_CUDA; break; }
        if (rep == 1) cudaEventRecord(e0, 0);
        if (mode == SG_PROBE_RED_DSM) {
            if (cudaLaunchKernelEx(&cfg, k_probe_red_dsm, (float2 *)acc, n, slice, magic, iters) != cudaSuccess) st = SG_ERR_CUDA;
            ops = (double)nclusters * cluster * 896.0 * iters;
        } else {
            const unsigned grid = (unsigned)sms * 8u;
            if (mode == SG_PROBE_RED8) k_probe_red8<<<grid, 256>>>((float2 *)acc, n, iters);
            else k_probe_red16<<<grid, 256>>>((float4 *)acc, n, iters);
            ops = (double)grid * 256.0 * iters;
        }
        if (rep == 1) cudaEventRecord(e1, 0);
    }
    if (st == SG_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        st = SG_ERR_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(acc);
    if (st == SG_OK && cudaGetLastError() != cudaSuccess) st = SG_ERR_CUDA;
    *out_seconds = st == SG_OK ? ms * 1e-3 : 0.0;
    *out_ops = st == SG_OK ? ops : 0.0;
    return st;
}
