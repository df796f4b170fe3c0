// Integer-pipe throughput microbenchmark: the peak behind the ALU roofline of
// the scan kernels (the paper has no counterpart; it is a measurement tool).
//
// Each thread runs eight independent chains of one instruction kind (LOP3,
// SHF, POPC or IMAD) written as inline PTX so that each step is exactly one
// instruction of that kind; enough warps are launched to fill every SM.  The
// kernel also reads the SM cycle counter and the global nanosecond timer at
// its start and end, so the clock the GPU actually ran at is measured on the
// device and the result can be given per SM per clock.
//
// The integer tensor-core forms that sm_103a offers are measured the same
// way, by warps issuing eight independent warp-wide mma.sync instructions
// per trip: signed 8-bit operands (m16n8k32, int32 accumulators) and 1-bit
// operands with AND + population count (m16n8k256 and m16n8k128).  The
// 1-bit form computes, per output, the number of set bits of (row AND
// column) over K bits: with a one-hot text row and a class-mask column that
// is the match count of Eq. 4's window over K/4 positions.  (The tcgen05
// instruction family has no integer kind on sm_103a: its i8 kind is not
// accepted for that target.)
#include "pm_internal.cuh"

namespace pm {
namespace {

// One warp-wide integer MMA, accumulating into d (OP 4: s8 m16n8k32; 5: b1
// AND-popc m16n8k256; 6: b1 AND-popc m16n8k128).  a, b: the lane's fragment
// registers (four of A, two of B; m16n8k128 uses two and one).
template <int OP>
__device__ __forceinline__ void mma_int(uint32_t (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    if constexpr (OP == 4) {
        asm volatile(
            "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    } else if constexpr (OP == 5) {
        asm volatile(
            "mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc {%0,%1,%2,%3}, "
            "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
            : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k128.row.col.s32.b1.b1.s32.and.popc {%0,%1,%2,%3}, "
            "{%4,%5}, {%6}, {%0,%1,%2,%3};"
            : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(b[0]));
    }
}

// Multiply-accumulates of one warp-wide MMA of kind OP (M x N x K).
constexpr double mma_macs(int op) { return op == 4 ? 16.0 * 8 * 32 : op == 5 ? 16.0 * 8 * 256 : 16.0 * 8 * 128; }

template <int OP>
__global__ void __launch_bounds__(256) k_mmapipe(uint32_t *out, uint32_t iters, uint32_t seed,
                                                 unsigned long long *clk)
{
    uint32_t a[4], b[2], d[8][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) a[j] = seed * (threadIdx.x + 1) + 0x9e3779b9u * (j + 1);
    b[0] = seed ^ threadIdx.x;
    b[1] = seed + 77u * threadIdx.x;
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int j = 0; j < 4; ++j) d[c][j] = 0u;
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long c0 = 0, t0 = 0;
    if (timer) {
        c0 = clock64();
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    }
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) mma_int<OP>(d[c], a, b);
    }
    if (timer) {
        unsigned long long c1 = clock64(), t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        clk[0] = c1 - c0;
        clk[1] = t1 - t0;
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc ^= d[c][j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

template <int OP>
__global__ void __launch_bounds__(256) k_intpipe(uint32_t *out, uint32_t iters, uint32_t seed,
                                                 unsigned long long *clk)
{
    uint32_t x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = seed * (threadIdx.x + 1) + 0x9e3779b9u * (j + 1);
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long c0 = 0, t0 = 0;
    if (timer) {
        c0 = clock64();
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    }
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t a = x[j], b = x[(j + 1) & 7], c = x[(j + 3) & 7];
            uint32_t r;
            if constexpr (OP == 0) {
                asm volatile("lop3.b32 %0, %1, %2, %3, 0xe8;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
            } else if constexpr (OP == 1) {
                asm volatile("shf.r.wrap.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
            } else if constexpr (OP == 2) {
                uint32_t p;
                asm volatile("popc.b32 %0, %1;" : "=r"(p) : "r"(b));
                r = a ^ p;  // the XOR keeps chains dependent; count only the POPC
            } else {
                asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
            }
            x[j] = r;
        }
    }
    if (timer) {
        unsigned long long c1 = clock64(), t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        clk[0] = c1 - c0;
        clk[1] = t1 - t0;
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) acc ^= x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace
}  // namespace pm

using namespace pm;

namespace pm {
namespace {

// The bounded barrier wait that any kernel waiting on an mbarrier (a bulk
// copy's completion) must use, on a barrier that receives its one arrival
// only if `arrive` is set: without it nothing completes the phase and the
// wait must give up after limit_ns.
// out[0] = 1 when the wait gave up, out[1] = 1 once the kernel returned.
__global__ void k_bounded_wait(uint64_t limit_ns, int arrive, uint32_t *out)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        dev::mbar_init(&bar, 1);
        dev::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (arrive) dev::mbar_arrive_expect_tx(&bar, 0);
        const bool ok = dev::mbar_wait_bounded(&bar, 0u, limit_ns);
        out[0] = ok ? 0u : 1u;
        out[1] = 1u;
    }
}

}  // namespace
}  // namespace pm

extern "C" {

pm_status pm_check_bounded_wait(uint64_t limit_ns, int32_t arrive, uint32_t *timed_out)
{
    if (!timed_out || limit_ns == 0 || limit_ns > 10000000000ull) {
        set_error("pm_check_bounded_wait: NULL output or limit outside 1 ns .. 10 s");
        return PM_E_ARG;
    }
    uint32_t *d = nullptr;
    pm_status rc = cuda_status(cudaMalloc(&d, 2 * sizeof(uint32_t)), "cudaMalloc");
    if (rc) return rc;
    uint32_t h[2] = {0u, 0u};
    rc = cuda_status(cudaMemset(d, 0, 2 * sizeof(uint32_t)), "cudaMemset");
    if (!rc) {
        k_bounded_wait<<<1, 32>>>(limit_ns, arrive ? 1 : 0, d);
        rc = cuda_status(cudaGetLastError(), "launch");
    }
    if (!rc) rc = cuda_status(cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost), "copy result");
    cudaFree(d);
    if (rc) return rc;
    if (h[1] != 1u) {
        set_error("pm_check_bounded_wait: the kernel did not finish");
        return PM_E_CUDA;
    }
    *timed_out = h[0];
    return PM_OK;
}

pm_status pm_measure_int_pipe(int32_t op, uint32_t iters, double *ops_per_s, double *sm_mhz,
                              double *ops_per_clk_per_sm)
{
    if (op < 0 || op > 6 || !ops_per_s || iters == 0) {
        set_error("pm_measure_int_pipe: op must be 0..6 (LOP3, SHF, POPC, IMAD, MMA s8, MMA b1 k256, "
                  "MMA b1 k128)");
        return PM_E_ARG;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void *fn = op == 0 ? (const void *)&k_intpipe<0>
                   : op == 1 ? (const void *)&k_intpipe<1>
                   : op == 2 ? (const void *)&k_intpipe<2>
                   : op == 3 ? (const void *)&k_intpipe<3>
                   : op == 4 ? (const void *)&k_mmapipe<4>
                   : op == 5 ? (const void *)&k_mmapipe<5> : (const void *)&k_mmapipe<6>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0);
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    uint32_t *out = nullptr;
    unsigned long long *clk = nullptr;
    pm_status rc = cuda_status(cudaMalloc(&out, (size_t)grid * 256 * 4 + 64), "cudaMalloc");
    if (rc) return rc;
    clk = (unsigned long long *)((char *)out + (size_t)grid * 256 * 4);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    uint32_t seed = 12345u;
    void *args[] = {(void *)&out, (void *)&iters, (void *)&seed, (void *)&clk};
    rc = cuda_status(cudaLaunchKernel(fn, dim3(grid), dim3(256), args, 0, 0), "warm-up launch");
    if (!rc) {
        cudaEventRecord(e0, 0);
        rc = cuda_status(cudaLaunchKernel(fn, dim3(grid), dim3(256), args, 0, 0), "timed launch");
        cudaEventRecord(e1, 0);
    }
    float ms = 0.f;
    unsigned long long hclk[2] = {0, 0};
    if (!rc) rc = cuda_status(cudaEventSynchronize(e1), "synchronize");
    if (!rc) {
        cudaEventElapsedTime(&ms, e0, e1);
        cudaMemcpy(hclk, clk, sizeof hclk, cudaMemcpyDeviceToHost);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (rc) return rc;
    // per-thread instructions, or for the MMA kinds 2 x M x N x K per warp instruction
    const double ops = op <= 3 ? (double)grid * 256.0 * iters * 8.0
                               : (double)grid * (256.0 / 32.0) * iters * 8.0 * 2.0 * mma_macs(op);
    *ops_per_s = ops / (ms * 1e-3);
    const double mhz = hclk[1] ? (double)hclk[0] / (double)hclk[1] * 1e3 : 0.0;
    if (sm_mhz) *sm_mhz = mhz;
    if (ops_per_clk_per_sm) *ops_per_clk_per_sm = mhz > 0 ? *ops_per_s / (sms * mhz * 1e6) : 0.0;
    return PM_OK;
}

}  // extern "C"
