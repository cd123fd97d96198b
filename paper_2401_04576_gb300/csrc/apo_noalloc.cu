// apo_vote_coarse_noalloc: full level-0 voting whose scratch memory is a fixed array
// compiled into the library instead of a workspace the caller allocates.
//
// Who needs it: code that may not allocate device memory when it votes, for example a
// process whose framework allocator owns the whole GPU memory budget, or a latency-bound
// loop where cudaMalloc / cudaFree (which can synchronise the device) are not allowed
// after start-up.  Such a caller still passes its inputs (hits) and its output buffer; the
// staging records, per-event hit counts, status word and vote histograms live here.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/apo.h"
#include "../../include/apo_diag.h"
#include "kernels.cuh"

using namespace apo;

namespace {

constexpr int kMaxEv = APO_NOALLOC_MAX_EVENTS;

constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
// layout of the fixed scratch array
constexpr size_t kOffStatus = 0;
constexpr size_t kOffNHits = 256;
constexpr size_t kOffHD = kOffNHits + al256(sizeof(int32_t) * kMaxEv);
constexpr size_t kOffHF = kOffHD + al256(sizeof(HitRecD) * kMaxEv * kHitCap);
constexpr size_t kOffHist = kOffHF + al256(sizeof(HitRecF) * kMaxEv * kHitCap);
constexpr size_t kOffActive = kOffHist + al256(sizeof(uint32_t) * kMaxEv * kHistBins);
constexpr size_t kOffDone = kOffActive + al256(sizeof(uint32_t) * kMaxEv * 8);
constexpr size_t kScratchBytes = kOffDone + al256(sizeof(int32_t) * kMaxEv);

// The scratch itself: one copy per device that loads this library, kept until the process
// exits.  In host code this name is only a stand-in for the symbol; the device address
// comes from cudaGetSymbolAddress below.
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

int err(int code, const char *what) {
    set_last_error(what);
    return code;
}

// Device address of the scratch array on the current device, looked up once per device.
int scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(APO_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(APO_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return err(APO_ECUDA, "cudaGetSymbolAddress of the fixed scratch failed");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return APO_OK;
}

}  // namespace

extern "C" int apo_vote_coarse_noalloc(const apo_geometry *g, const apo_hits *hits, int32_t precision,
                                       int32_t *votes_out, void *stream) {
    if (!g || !hits || !votes_out) return err(APO_EINVAL, "geometry, hits and votes_out must be non-NULL");
    if (hits->n_events < 0) return err(APO_EINVAL, "n_events < 0");
    if (hits->n_events > kMaxEv) {
        char msg[160];
        std::snprintf(msg, sizeof(msg),
                      "apo_vote_coarse_noalloc: %d events exceed the fixed scratch limit of %d",
                      hits->n_events, kMaxEv);
        return err(APO_EINVAL, msg);
    }
    if (hits->n_events > 0 && (!hits->offsets || !hits->wire_id || !hits->drift))
        return err(APO_EINVAL, "hits arrays must be non-NULL");
    if (precision != APO_F64 && precision != APO_F32 && precision != APO_F64_FILTERED &&
        precision != APO_F64_MID && precision != APO_F64_EXACT)
        return err(APO_EINVAL, "bad precision");
    int gdev = -1;
    const DevGeom *dg = geometry_device_tables(g, &gdev);
    if (precision == APO_F64_MID && !dg->sincos_mid)
        return err(APO_EINVAL, "APO_F64_MID needs the grid's sincos_mid table");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != gdev)
        return err(APO_EINVAL, "geometry is not on the current device");
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != APO_OK) return rc;
    const int ne = hits->n_events;
    if (ne == 0) return APO_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char *b = static_cast<unsigned char *>(base);
    unsigned *status = reinterpret_cast<unsigned *>(b + kOffStatus);
    int32_t *nh = reinterpret_cast<int32_t *>(b + kOffNHits);
    HitRecD *hd = reinterpret_cast<HitRecD *>(b + kOffHD);
    HitRecF *hf = reinterpret_cast<HitRecF *>(b + kOffHF);
    uint32_t *hist = reinterpret_cast<uint32_t *>(b + kOffHist);
    uint32_t *active = reinterpret_cast<uint32_t *>(b + kOffActive);
    int32_t *done = reinterpret_cast<int32_t *>(b + kOffDone);
    // the array keeps the previous call's contents: clear what the kernels accumulate into
    cudaError_t e = cudaMemsetAsync(status, 0, 256, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)ne * kHistBins, s);
    if (e != cudaSuccess) return err(APO_ECUDA, cudaGetErrorString(e));
    launch_stage(*dg, ne, hits->offsets, hits->wire_id, hits->drift, hd, hf, nh, active, done, status, s);
    launch_vote_coarse(*dg, precision, 0, ne, hd, hf, nh, votes_out, hist, status, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return err(APO_ECUDA, cudaGetErrorString(e));
    return APO_OK;
}

// The status bits published in apo.h are the kernels' own status bits.
static_assert(APO_STATUS_TIMEOUT == ST_TIMEOUT && APO_STATUS_BADHIT == ST_BADHIT &&
                  APO_STATUS_TOOMANY == ST_TOOMANY && APO_STATUS_BADOFFS == ST_BADOFFS,
              "status bits");

extern "C" int apo_vote_coarse_noalloc_status(uint32_t *flags_out, void *stream) {
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != APO_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, static_cast<unsigned char *>(base) + kOffStatus, sizeof(unsigned),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return err(APO_ECUDA, cudaGetErrorString(e));
    if (flags_out) *flags_out = h;
    if (h & ST_TIMEOUT) return err(APO_ETIMEOUT, "a device wait ran out of its poll limit");
    if (h & (ST_BADHIT | ST_TOOMANY | ST_BADOFFS))
        return err(APO_EINVAL, "malformed event(s) in the last apo_vote_coarse_noalloc call (zero votes)");
    return APO_OK;
}

extern "C" int apo_diag_noalloc_wait_timeout(int32_t limit_polls, void *stream) {
    if (limit_polls < 1) return err(APO_EINVAL, "limit_polls < 1");
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != APO_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned *status = reinterpret_cast<unsigned *>(static_cast<unsigned char *>(base) + kOffStatus);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return err(APO_ECUDA, cudaGetErrorString(e));
    launch_wait_never(limit_polls, status, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return err(APO_ECUDA, cudaGetErrorString(e));
    return APO_OK;
}
