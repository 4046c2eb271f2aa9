// crk_fma_peak: the device's measured fused-multiply-add throughput, the
// denominator of the pair passes' roofline fractions (FP32 for the mixed
// form, FP64 for the plain form, whose rate on this part is a small fraction
// of the FP32 rate and is measured rather than taken from a data sheet).
//
// Every thread runs kChains independent FMA chains (enough to cover the FMA
// pipe's latency) for kIters iterations; the grid fills every SM with
// resident blocks.  The chains' results feed a store that never happens (a
// comparison with a value they cannot reach), so the compiler keeps the work.
#include "sim.h"

namespace crk {

namespace {

constexpr int kT = 256;
constexpr int kChains = 8;
constexpr int kIters = 4096;

template <typename R>
__global__ void __launch_bounds__(kT) fma_chains_k(R a, R b, R *sink)
{
    R acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (R)(threadIdx.x + c) * (R)1e-3;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
    }
    R s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == (R)-12345.0) sink[0] = s;  // unreachable for a in (0, 1), b > 0
}

template <typename R>
int measure(double *tflops, cudaStream_t st)
{
    int dev = 0, sms = 0, per_sm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chains_k<R>, kT, 0));
    const unsigned grid = (unsigned)(sms * (per_sm > 0 ? per_sm : 1) * 4);
    const R a = (R)0.999999, b = (R)1e-7;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    fma_chains_k<R><<<grid, kT, 0, st>>>(a, b, nullptr);  // warm-up (clocks up, code loaded)
    cudaEventRecord(e0, st);
    const int reps = 3;
    for (int r = 0; r < reps; ++r) fma_chains_k<R><<<grid, kT, 0, st>>>(a, b, nullptr);
    cudaEventRecord(e1, st);
    note_launches(1 + reps);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(err);
    CK(cudaGetLastError());
    const double flop = 2.0 * (double)grid * kT * kChains * (double)kIters * reps;
    *tflops = ms > 0.f ? flop / (ms * 1e-3) / 1e12 : 0.0;
    return CRK_OK;
}

}  // namespace

}  // namespace crk

extern "C" int crk_fma_peak(int precision, double *tflops, void *cuda_stream)
{
    using namespace crk;
    if (!tflops) return fail(CRK_EINVAL, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (precision == CRK_MIXED) return measure<float>(tflops, st);
    if (precision == CRK_FP64) return measure<double>(tflops, st);
    return fail(CRK_EINVAL, "precision must be CRK_FP64 or CRK_MIXED");
}
