// rbe_noalloc.cu -- the Fourier part of one RBE evaluation for callers that
// cannot allocate device memory.
//
// Who needs this: an MD engine that hands all device memory to its own pool at
// start-up and forbids plugins from calling cudaMalloc; a latency-bound loop
// where cudaMalloc's implicit device-wide synchronisation would stall the
// other streams.  Such a
// caller cannot create an rbe handle (rbe_create allocates the workspace), so
// this entry point keeps its scratch in one file-scope device array instead:
// the sampling table, the per-chunk partial structure factors, the per-k
// coefficients and the per-chunk charge sums.  The caller passes only the
// particles and the outputs.
//
// The array is g_rbe_noalloc_scratch (kNoAllocScratchBytes = 4 MiB).  Every GPU
// that loads librbe holds it until the process exits.  The host never uses the
// symbol's name as a pointer: on the first call on a device, with that device
// current, cudaGetSymbolAddress gives its device address, which is cached per
// device and passed to the kernels.
//
// All calls share the one array and each call overwrites every part it later
// reads (nothing has to start at zero), so the contents left by the previous
// call never matter.  Calls whose work overlaps on the GPU (for example on two
// streams at once) race on the array and give wrong results: serialise them.
#include <cmath>
#include <mutex>

#include "rbe.h"
#include "rbe_internal.cuh"

namespace rbe {
namespace noalloc {

constexpr size_t kNoAllocScratchBytes = 4u << 20;     // 4 MiB per device
constexpr int kMaxP = 1024;                           // wave vectors per call
constexpr int kMaxTable = 4096;                       // table entries (M <= 2047)
constexpr int kMaxChunk = 1 << 16;                    // particles per chunk
constexpr int kMaxDevices = 64;
constexpr int kThreads = 128;
constexpr int kStageN = 512;
constexpr float kTwoPiOver2p32 = 1.4629180792671596e-09f;

static __device__ __align__(256) unsigned char g_rbe_noalloc_scratch[kNoAllocScratchBytes];

// Byte offsets of the scratch regions for one call (all 256-byte aligned).
struct Layout {
    size_t table, ksamp, kab, eterm, qpart, part, end;
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline Layout layout(int P, int nchunk) {
    Layout L;
    L.table = 0;
    L.ksamp = align256(L.table + sizeof(uint64_t) * kMaxTable);
    L.kab = align256(L.ksamp + sizeof(int4) * P);
    L.eterm = align256(L.kab + sizeof(float2) * P);
    L.qpart = align256(L.eterm + sizeof(double) * P);
    L.part = align256(L.qpart + sizeof(double2) * nchunk);
    L.end = L.part + sizeof(float2) * (size_t)nchunk * P;
    return L;
}

struct Args {
    uint64_t seed, step;
    uint32_t stream;
    int P, M, n, chunk, nchunk;
    float fx_hi, fx_lo;
    double invL, coef_scale, self_coef, bg_coef;
    Layout L;
};

__device__ __forceinline__ uint32_t na_fixed(float x, float hi, float lo) {
    const float p = x * hi;
    const float e = fmaf(x, hi, -p);
    float corr = fmaf(x, lo, e);
    const float pr = rintf(p);
    corr += (p - pr);
    return (uint32_t)(unsigned long long)((long long)pr + __float2ll_rn(corr));
}

__device__ __forceinline__ int na_lookup(const uint64_t* T, int n, uint32_t w) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((uint64_t)w < T[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Per-chunk partial structure factors (the variant of the structure-factor
// kernel whose partials live in the static scratch), the k-batch, and the
// chunk's charge sums.
__global__ void __launch_bounds__(kThreads)
k_na_rho(Args a, const float4* __restrict__ pos_q, unsigned char* __restrict__ scratch,
         int* __restrict__ err) {
    __shared__ uint4 sp[kStageN];
    const uint64_t* T = (const uint64_t*)(scratch + a.L.table);
    int4* ksamp = (int4*)(scratch + a.L.ksamp);
    double2* qpart = (double2*)(scratch + a.L.qpart);
    float2* part = (float2*)(scratch + a.L.part);
    const int c = blockIdx.x;
    const int l = blockIdx.y * kThreads + threadIdx.x;
    const bool active = l < a.P;
    const int first = c * a.chunk;
    const int count = max(0, min(a.chunk, a.n - first));
    int4 m = make_int4(0, 0, 0, 0);
    if (active) {
        const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
        const int nt = 2 * a.M + 1;
        bool ok = false;
        for (int at = 0; at < kMaxAttempts && !ok; ++at) {
            const uint4 w = philox4x32_10(
                make_uint4((uint32_t)l, (uint32_t)at, (uint32_t)a.step, (a.stream << 8) | 0x01u),
                key);
            m = make_int4(na_lookup(T, nt, w.x) - a.M, na_lookup(T, nt, w.y) - a.M,
                          na_lookup(T, nt, w.z) - a.M, at + 1);
            ok = (m.x | m.y | m.z) != 0;
        }
        if (!ok) {
            atomicOr(err, kErrSampler);
            m = make_int4(1, 0, 0, kMaxAttempts + 1);
        }
        if (c == 0) ksamp[l] = m;
    }
    // FP32 sums over one staged pass (at most kStageN terms), carried in FP64
    // across passes, so that the rounding does not grow with the chunk size
    double red = 0.0, imd = 0.0;
    double qs = 0.0, q2s = 0.0;
    for (int base = 0; base < count; base += kStageN) {
        const int cnt = min(kStageN, count - base);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const float4 p = pos_q[first + base + t];
            latch_any(!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w)), err,
                      kErrNonfinite);
            sp[t] = make_uint4(na_fixed(p.x, a.fx_hi, a.fx_lo), na_fixed(p.y, a.fx_hi, a.fx_lo),
                               na_fixed(p.z, a.fx_hi, a.fx_lo), __float_as_uint(p.w));
            if (blockIdx.y == 0) {
                qs += (double)p.w;
                q2s += (double)p.w * (double)p.w;
            }
        }
        __syncthreads();
        if (active) {
            float re = 0.f, im = 0.f;
            for (int j = 0; j < cnt; ++j) {
                const uint4 p = sp[j];
                const uint32_t ph = (uint32_t)m.x * p.x + (uint32_t)m.y * p.y + (uint32_t)m.z * p.z;
                float sn, cs;
                __sincosf((float)(int32_t)ph * kTwoPiOver2p32, &sn, &cs);
                const float q = __uint_as_float(p.w);
                re = fmaf(q, cs, re);
                im = fmaf(q, sn, im);
            }
            red += (double)re;
            imd += (double)im;
        }
    }
    // the chunk's partial, rounded once to FP32 (a relative 2^-24 of the
    // chunk's sum; the chunks are then added in FP64)
    if (active) part[(size_t)c * a.P + l] = make_float2((float)red, (float)imd);
    if (blockIdx.y == 0) {
        __shared__ double sq[kThreads], sq2[kThreads];
        sq[threadIdx.x] = qs;
        sq2[threadIdx.x] = q2s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double A = 0.0, B = 0.0;
            for (int t = 0; t < kThreads; ++t) { A += sq[t]; B += sq2[t]; }
            qpart[c] = make_double2(A, B);
        }
    }
}

// FP64 sum of the chunk partials per k (fixed order), force coefficients and
// energy terms.
__global__ void k_na_finalize(Args a, unsigned char* __restrict__ scratch) {
    const int4* ksamp = (const int4*)(scratch + a.L.ksamp);
    float2* kab = (float2*)(scratch + a.L.kab);
    double* eterm = (double*)(scratch + a.L.eterm);
    const float2* part = (const float2*)(scratch + a.L.part);
    const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (l >= a.P) return;
    double re = 0.0, im = 0.0;
    for (int c = lane; c < a.nchunk; c += 32) {
        const float2 v = part[(size_t)c * a.P + l];
        re += (double)v.x;
        im += (double)v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
        const int4 m = ksamp[l];
        const double tp = 2.0 * M_PI * a.invL;
        const double k2 = tp * tp * ((double)m.x * m.x + (double)m.y * m.y + (double)m.z * m.z);
        const double coef = a.coef_scale / k2;
        kab[l] = make_float2((float)(coef * im), (float)(coef * re));
        eterm[l] = 0.5 * coef * (re * re + im * im);
    }
}

// Fourier force per particle, in the caller's order.
__global__ void __launch_bounds__(kThreads)
k_na_force(Args a, const float4* __restrict__ pos_q, const unsigned char* __restrict__ scratch,
           float4* __restrict__ F_out) {
    constexpr int kKT = 256;
    __shared__ uint4 km[kKT];
    __shared__ float4 kf[kKT];
    const int4* ksamp = (const int4*)(scratch + a.L.ksamp);
    const float2* kab = (const float2*)(scratch + a.L.kab);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < a.n;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    if (active) p = pos_q[i];
    const uint32_t sx = na_fixed(p.x, a.fx_hi, a.fx_lo), sy = na_fixed(p.y, a.fx_hi, a.fx_lo),
                   sz = na_fixed(p.z, a.fx_hi, a.fx_lo);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int base = 0; base < a.P; base += kKT) {
        const int cnt = min(kKT, a.P - base);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            const int4 m = ksamp[base + k];
            const float2 ab = kab[base + k];
            km[k] = make_uint4((uint32_t)m.x, (uint32_t)m.y, (uint32_t)m.z, __float_as_uint(ab.y));
            kf[k] = make_float4((float)m.x, (float)m.y, (float)m.z, ab.x);
        }
        __syncthreads();
        if (active) {
            for (int k = 0; k < cnt; ++k) {
                const uint4 mk = km[k];
                const float4 f = kf[k];
                const uint32_t ph = mk.x * sx + mk.y * sy + mk.z * sz;
                float sn, cs;
                __sincosf((float)(int32_t)ph * kTwoPiOver2p32, &sn, &cs);
                const float g = fmaf(cs, f.w, -sn * __uint_as_float(mk.w));
                fx = fmaf(g, f.x, fx);
                fy = fmaf(g, f.y, fy);
                fz = fmaf(g, f.z, fz);
            }
        }
    }
    if (active) {
        const float sc = -p.w * (float)(2.0 * M_PI) * (float)a.invL;
        F_out[i] = make_float4(sc * fx, sc * fy, sc * fz, 0.f);
    }
}

// Fourier energy: estimator terms minus self and background terms.
__global__ void k_na_energy(Args a, const unsigned char* __restrict__ scratch,
                            double* __restrict__ E_out) {
    const double* eterm = (const double*)(scratch + a.L.eterm);
    const double2* qpart = (const double2*)(scratch + a.L.qpart);
    __shared__ double se[256], sq[256], sq2[256];
    double e = 0.0, q = 0.0, q2 = 0.0;
    for (int l = threadIdx.x; l < a.P; l += blockDim.x) e += eterm[l];
    for (int c = threadIdx.x; c < a.nchunk; c += blockDim.x) {
        q += qpart[c].x;
        q2 += qpart[c].y;
    }
    se[threadIdx.x] = e; sq[threadIdx.x] = q; sq2[threadIdx.x] = q2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            se[threadIdx.x] += se[threadIdx.x + o];
            sq[threadIdx.x] += sq[threadIdx.x + o];
            sq2[threadIdx.x] += sq2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        E_out[0] = se[0] - a.self_coef * sq2[0] - 0.5 * a.bg_coef * sq[0] * sq[0];
}

__global__ void k_na_clear_err(int* err) { *err = 0; }

// ------------------------------------------------------------------ host
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (cached).
cudaError_t scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_rbe_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (unsigned char*)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace noalloc
}  // namespace rbe

namespace rbe {
void set_last_error_message(const char* msg);   // rbe_api.cu: read by rbe_last_error(NULL)
}

namespace {
rbe_status na_fail(rbe_status s, const char* msg) {
    rbe::set_last_error_message(msg);
    return s;
}
}  // namespace

extern "C" rbe_status rbe_fourier_forces_noalloc(const rbe_params* p, int32_t n,
                                                 const float* pos_q, uint64_t step,
                                                 float* F_out, double* E_out,
                                                 void* cuda_stream) {
    using namespace rbe::noalloc;
    if (!p) return na_fail(RBE_ERR_ARG, "params is NULL");
    if (n < 0 || (n > 0 && (!pos_q || !F_out))) return na_fail(RBE_ERR_ARG, "bad n or null buffer");
    if (!(p->box > 0.0) || !(p->alpha > 0.0) || !std::isfinite(p->box) ||
        !std::isfinite(p->alpha))
        return na_fail(RBE_ERR_ARG, "box and alpha must be finite and > 0");
    if (!std::isfinite(p->coulomb_prefactor))
        return na_fail(RBE_ERR_ARG, "coulomb_prefactor must be finite");
    if (p->sampler != RBE_SAMPLER_EXACT)
        return na_fail(RBE_ERR_ARG, "the no-allocation entry point draws the k-batch with the "
                                    "exact sampler only (sampler must be RBE_SAMPLER_EXACT)");
    if (p->P < 1 || p->P > kMaxP) return na_fail(RBE_ERR_ARG, "P must be in [1, 1024] for the no-allocation entry point");
    const double L = p->box;
    const int M = (int)std::ceil(std::sqrt(p->alpha * L * L * (64.0 * std::log(2.0))) / M_PI);
    if (2 * M + 1 > kMaxTable) return na_fail(RBE_ERR_ARG, "alpha L^2 too large: the sampling table exceeds 4096 entries");
    {
        const double H = std::sqrt(p->alpha * L * L / M_PI);
        if (H * H * H < 2.0) return na_fail(RBE_ERR_ARG, "alpha L^2 too small: k = 0 would dominate the sampler");
    }
    // chunk: smallest power of two >= 512 whose partials fit in the scratch
    int chunk = 512, nchunk = 1;
    for (;;) {
        nchunk = n > 0 ? (n + chunk - 1) / chunk : 1;
        if (layout(p->P, nchunk).end <= kNoAllocScratchBytes - 256) break;
        if (chunk >= kMaxChunk) return na_fail(RBE_ERR_ARG, "n * P too large for the 4 MiB scratch of the no-allocation entry point");
        chunk <<= 1;
    }
    const Layout Lay = layout(p->P, nchunk);
    if (n == 0 && !E_out) return RBE_OK;              // nothing to compute
    // sampling table: the same FP64 arithmetic as rbe_create, on the stack
    uint64_t table[kMaxTable];
    double Z = 0.0;
    {
        const double a = (M_PI * M_PI) / (p->alpha * L * L);
        const int nt = 2 * M + 1;
        for (int j = 0; j < nt; ++j) {
            const long long d = (long long)(j - M);
            Z += std::exp(-(a * (double)(d * d)));
        }
        double cum = 0.0;
        for (int j = 0; j < nt; ++j) {
            const long long d = (long long)(j - M);
            cum += std::exp(-(a * (double)(d * d)));
            if (j == nt - 1) {
                table[j] = 4294967296ull;
            } else {
                double f = std::floor((cum / Z) * 4294967296.0);
                if (f > 4294967295.0) f = 4294967295.0;
                table[j] = (uint64_t)f;
            }
        }
    }
    const double S = Z * Z * Z - 1.0;
    const double V = L * L * L;
    Args a{};
    a.seed = p->seed;
    a.step = step;
    a.stream = p->stream;
    a.P = p->P;
    a.M = M;
    a.n = n;
    a.chunk = chunk;
    a.nchunk = nchunk;
    const double scale = 4294967296.0 / L;
    a.fx_hi = (float)scale;
    a.fx_lo = (float)(scale - (double)a.fx_hi);
    a.invL = 1.0 / L;
    a.coef_scale = p->coulomb_prefactor * (S / (double)p->P) * 4.0 * M_PI / V;
    a.self_coef = p->coulomb_prefactor * std::sqrt(p->alpha / M_PI);
    a.bg_coef = p->coulomb_prefactor * M_PI / (V * p->alpha);
    a.L = Lay;

    unsigned char* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return na_fail(RBE_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the sampler's error word: the last 256 bytes of the array, outside the layout
    int* err = (int*)(scratch + kNoAllocScratchBytes - 256);
    e = cudaMemcpyAsync(scratch + Lay.table, table, sizeof(uint64_t) * (2 * M + 1),
                        cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return na_fail(RBE_ERR_CUDA, cudaGetErrorString(e));
    k_na_clear_err<<<1, 1, 0, st>>>(err);
    const int ltiles = (p->P + kThreads - 1) / kThreads;
    k_na_rho<<<dim3(nchunk, ltiles), kThreads, 0, st>>>(a, (const float4*)pos_q, scratch, err);
    k_na_finalize<<<(p->P * 32 + 255) / 256, 256, 0, st>>>(a, scratch);
    if (n > 0)
        k_na_force<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(a, (const float4*)pos_q,
                                                                        scratch, (float4*)F_out);
    if (E_out) k_na_energy<<<1, 256, 0, st>>>(a, scratch, E_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(RBE_ERR_CUDA, cudaGetErrorString(e));
    // The sampler's error word comes back on the caller's stream, behind the
    // kernels; one synchronisation of that stream (not of the device) then
    // covers it and the table copy, which reads host stack memory.
    int h_err = 0;
    e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return na_fail(RBE_ERR_CUDA, cudaGetErrorString(e));
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return na_fail(RBE_ERR_CUDA, cudaGetErrorString(e));
    if (h_err & rbe::kErrSampler)
        return na_fail(RBE_ERR_SAMPLER, "a k-sample drew (0,0,0) on 32 attempts in a row");
    if (h_err & rbe::kErrNonfinite)
        return na_fail(RBE_ERR_NONFINITE, "a position or charge was NaN or infinite");
    return RBE_OK;
}
