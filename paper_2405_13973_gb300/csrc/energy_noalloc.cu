// energy_noalloc.cu -- pt_energy_noalloc: the rotating-frame energy with the
// exact direct Coulomb sum, using only memory that exists before the call.
//
// pt_energy(NULL plan, ...) obtains its scratch (a packed copy of the
// positions, the field, the potential and the reduction partials) from
// cudaMalloc on every call.  Some callers cannot do that: real-time loops
// that must not pay cudaMalloc's implicit device synchronisation in the
// middle of a run, and host programs whose device memory is reserved up
// front by their own allocator.  This entry point serves them: its scratch
// is the file-scope array below, which every GPU that loads the library
// holds from module load until process exit.  The call ends with a copy of
// the four results to the host and a synchronisation of the stream.
//
// Contract of the scratch array:
//   * it is sized for at most kNoAllocMaxIons ions; larger states are
//     rejected with PT_ERR_ARG before any work is queued;
//   * every call writes every scratch element it later reads (the position
//     copy, the field and potential of all n ions, all reduction partials),
//     so nothing left by an earlier call can leak into a result and nothing
//     needs to be cleared;
//   * all calls on one device share the one array: calls whose work
//     overlaps on the GPU (different streams, or different host threads)
//     race on it and give undefined results.  Serialise them.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace {

constexpr int64_t kNoAllocMaxIons = 65536;
constexpr int kPartialBlocks = 256;  // matches the energy reduction's block count
// positions (3n), field (3n), potential (n), 4 results, 3 partials per block
constexpr int64_t kScratchDoubles = 7 * kNoAllocMaxIons + 4 + 3 * kPartialBlocks;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device with that device current (the host-side symbol is only a
// stand-in, never a device address).  This set-up runs in the first call on
// a device; the lookup may load the module, so that first call should come
// before any stream capture on the device.
cudaError_t scratch_on_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

int status_of(cudaError_t e) { return e == cudaSuccess ? PT_OK : PT_ERR_CUDA; }

}  // namespace

extern "C" int pt_energy_noalloc(const pt_state* st, const pt_trap* trap, double* out,
                                 void* stream) {
    if (!st || !trap || !out || st->n < 1 || !st->x || !st->y || !st->z || !st->vx ||
        !st->vy || !st->vz || !st->q || trap->charge == 0.0)
        return PT_ERR_ARG;
    if (st->n > kNoAllocMaxIons) return PT_ERR_ARG;
    double* base = nullptr;
    cudaError_t e = scratch_on_current_device(&base);
    if (e != cudaSuccess) return status_of(e);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = st->n;
    double* pos = base;
    double* E = pos + 3 * n;
    double* phi = E + 3 * n;
    double* dout = phi + n;  // 4 results followed by the reduction partials
    e = cudaMemcpyAsync(pos, st->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pos + n, st->y, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pos + 2 * n, st->z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = pt::launch_direct(n, pos, st->q, E, phi, s);
    const double kz = trap->mass * trap->omega_z * trap->omega_z / trap->charge;
    if (e == cudaSuccess) e = pt::launch_energy_parts(n, *st, *trap, kz, phi, dout, s);
    double h[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, dout, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return status_of(e);
    out[0] = h[0];
    out[1] = h[1];
    out[2] = h[2];
    out[3] = h[0] + h[1] + h[2];
    return PT_OK;
}
