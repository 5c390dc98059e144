// fricp_eval_pass_static: the fused correspondence pass of fricp_eval_pass for
// callers that must not allocate device memory. Everything the pass needs
// beyond the caller's input and output lives in one file-scope device array
// (g_scratch below), which each GPU that loads the library keeps until the
// process exits.
//
// Who needs this: a caller that has already given all device memory to another
// allocator (a framework's caching allocator that reserved the device), a
// latency-critical loop where cudaMalloc / cudaFree would synchronize the
// device, or a real-time or certified deployment that forbids allocation after
// start-up.
#include <atomic>
#include <cmath>
#include <cstring>

#include "host_common.cuh"

namespace {

using fricp::PairState;

constexpr int64_t kStaticMaxPoints = 32768;                        // largest m accepted
constexpr int kStaticTiles = (int)(kStaticMaxPoints / fricp::kBlock);
constexpr size_t kStateBytes = 16384;                               // >= sizeof(PairState)
constexpr size_t kTBytes = 256;                                     // 12 doubles, then the input flag
constexpr size_t kPartialBytes = sizeof(double) * kStaticTiles * fricp::kMaxSums;
constexpr size_t kPrevBytes = sizeof(int) * kStaticMaxPoints;
constexpr size_t kSrcBytes = sizeof(float4) * kStaticMaxPoints;
constexpr size_t kOffT = kStateBytes;
constexpr size_t kOffFlag = kOffT + 128;                            // int: a source coordinate is NaN/Inf
constexpr size_t kOffPartial = kOffT + kTBytes;
constexpr size_t kOffPrev = kOffPartial + kPartialBytes;
constexpr size_t kOffSrc = kOffPrev + kPrevBytes;
constexpr size_t kScratchBytes = kOffSrc + kSrcBytes;               // about 0.7 MB
static_assert(sizeof(PairState) <= kStateBytes, "state region too small");
static_assert(kOffPartial % 256 == 0 && kOffPrev % 256 == 0 && kOffSrc % 256 == 0,
              "region alignment");

// The scratch of every call. Host code must not pass this name to a kernel: on
// the host it is only a stand-in; its device address comes from
// cudaGetSymbolAddress (see scratch_address).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
// Device address of g_scratch per device, looked up by the first call on that
// device. It belongs to that device's primary context: after cudaDeviceReset
// the cached address is stale and must not be used, so a process that resets
// a device must not call this entry point on that device again.
std::atomic<char *> g_addr[kMaxDevices];

// Source points in caller order as float4 (.w = index); no sort, no allocation.
// Sets *bad when a coordinate is NaN or Inf (the allocating pass rejects such
// input the same way).
__global__ void k_pack_source(const float *__restrict__ p, int m, float4 *__restrict__ out, int *bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) {
        const float x = p[3 * i], y = p[3 * i + 1], z = p[3 * i + 2];
        if (!isfinite(x) || !isfinite(y) || !isfinite(z)) atomicOr(bad, 1);
        out[i] = make_float4(x, y, z, __int_as_float(i));
    }
}

fricp_status static_fail(fricp_status s, const char *msg) {
    fricp::set_last_error(msg);
    return s;
}

// One-time set-up on the current device: the device address of g_scratch.
fricp_status scratch_address(char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(FRICP_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return static_fail(FRICP_EINVAL, "device index out of range");
    char *addr = g_addr[dev].load(std::memory_order_acquire);
    if (addr == nullptr) {   // concurrent first calls look up the same address
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess || ptr == nullptr)
            return static_fail(FRICP_ECUDA, "cudaGetSymbolAddress(g_scratch) failed");
        addr = (char *)ptr;
        g_addr[dev].store(addr, std::memory_order_release);
    }
    *out = addr;
    return FRICP_OK;
}

}  // namespace

extern "C" fricp_status fricp_eval_pass_static(const fricp_target *target, const float *p_xyz_dev, int64_t m,
                                               int32_t variant, const double *T_normalized, double nu,
                                               double scale, const double *center, void *stream, double *out) {
    if (!target || !p_xyz_dev || !T_normalized || !out) return static_fail(FRICP_EINVAL, "NULL argument");
    if (m < 1 || m > kStaticMaxPoints)
        return static_fail(FRICP_EINVAL, "m must be in 1..32768 for fricp_eval_pass_static");
    if (variant < FRICP_P2P_AA || variant > FRICP_P2PL_AA) return static_fail(FRICP_EINVAL, "unknown variant");
    const fricp::TargetDev &td = *fricp::target_dev(target);
    if (fricp::variant_p2pl(variant) && !td.has_normals)
        return static_fail(FRICP_EUNSUPPORTED, "point-to-plane needs target normals");
    if (!(scale > 0.0)) return static_fail(FRICP_EINVAL, "scale must be > 0");
    if (fricp::variant_robust(variant) && !(nu > 0.0)) return static_fail(FRICP_EINVAL, "nu must be > 0");
    char *base = nullptr;
    fricp_status st = scratch_address(&base);
    if (st != FRICP_OK) return st;
    const cudaStream_t s = (cudaStream_t)stream;
    PairState *st_dev = reinterpret_cast<PairState *>(base);
    double *T_dev = reinterpret_cast<double *>(base + kOffT);
    double *partial = reinterpret_cast<double *>(base + kOffPartial);
    int *prev = reinterpret_cast<int *>(base + kOffPrev);
    int *bad_dev = reinterpret_cast<int *>(base + kOffFlag);
    float4 *src = reinterpret_cast<float4 *>(base + kOffSrc);
    const int ntiles = (int)((m + fricp::kBlock - 1) / fricp::kBlock);

    // Host-side state image: the same initial state as fricp_eval_pass.
    fricp_params prm;
    fricp_params_default(variant, &prm);
    const double c[3] = {center ? center[0] : 0.0, center ? center[1] : 0.0, center ? center[2] : 0.0};
    PairState h = fricp::host::initial_state(prm, m, ntiles, scale, c, 1.0, 0);
    h.nu = fricp::variant_robust(variant) ? nu : 1.0;
    double T12[12];
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) T12[3 * r + k] = T_normalized[4 * r + k];
        T12[9 + r] = T_normalized[4 * r + 3];
    }
    // Every region the pass reads is rewritten here, so nothing from the last
    // call leaks in: the whole state (its last-block counter included), T, the
    // input flag, the correspondences (-1: none) and the packed source. Tile
    // records are written by the pass before they are read.
    cudaError_t e = cudaMemcpyAsync(st_dev, &h, sizeof(h), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(T_dev, T12, sizeof(T12), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad_dev, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(prev, 0xff, sizeof(int) * m, s);
    if (e == cudaSuccess) {
        k_pack_source<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(p_xyz_dev, (int)m, src, bad_dev);
        fricp::counters().launches += 1;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = fricp::launch_setup_eval_xi(st_dev, T_dev, s);
    fricp::StepArgs a;
    a.st = st_dev;
    a.ix = fricp::make_index(td);
    a.src = src;
    a.prev = prev;
    a.partial = partial;
    a.resid = nullptr;
    a.trace = nullptr;
    if (e == cudaSuccess) e = fricp::launch_step(a, variant, fricp::PREC_FP64, ntiles, s, nullptr, FRICP_SEARCH_QUERY);   // a cold pass
    PairState r;
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&r, st_dev, sizeof(r), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, bad_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return static_fail(FRICP_ECUDA, cudaGetErrorString(e));
    fricp::counters().h2d += sizeof(h) + sizeof(T12);
    fricp::counters().d2h += sizeof(r) + sizeof(int);
    if (bad) return static_fail(FRICP_EINVAL, "p_xyz has NaN or Inf");
    if (r.nn_overflow) return static_fail(FRICP_EOVERFLOW, "closest-point search stack overflow");
    for (int i = 0; i < 48; ++i) out[i] = r.eval_out[i];
    if (r.status == FRICP_EDEGENERATE) return static_fail(FRICP_EDEGENERATE, "degenerate alignment problem");
    return FRICP_OK;
}
