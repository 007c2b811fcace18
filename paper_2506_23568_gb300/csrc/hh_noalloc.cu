// Direct BPA with a fixed, statically reserved device workspace.
//
// bpa_form_image obtains its workspace (trajectory copy, twiddle table, range
// profiles, counters) with stream-ordered device allocation on every call.
// Some callers cannot allocate at the moment they want an image: code running
// under a device-memory budget that was fixed at start-up, or a caller that has
// already handed every free byte of the device to its own memory pool.  This
// entry point serves them: its workspace is one file-scope __device__ array of
// fixed size, reserved when this translation unit's module is loaded, and the
// call itself performs no allocation of device or host memory.
//
// The array's address is looked up once per device (with that device current)
// on the first call, which may also load the module.  The cached address does
// not survive cudaDeviceReset (or the destruction of the device's primary
// context).  There is one array per device, so two calls that overlap in time on
// the same device (different streams or host threads) race on it.

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "hh_internal.h"
#include "hhffbp.h"

namespace {

static __device__ __align__(256) unsigned char g_bpa_scratch[HH_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// W[q] = exp(+j pi q / n_fft), q in [0, 2 n_fft): the range-compression
// twiddles, computed in FP64 on the device and rounded to FP32.
__global__ void k_noalloc_twiddles(float2* w, int n_fft) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 2 * n_fft) return;
    double s, c;
    sincospi((double)q / (double)n_fft, &s, &c);
    w[q] = make_float2((float)c, (float)s);
}

// Device address of the workspace on the current device (looked up once).
int scratch_of_current_device(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return hh::note_cuda_error((int)e);
    if (dev < 0 || dev >= kMaxDevices) return HH_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bpa_scratch);
        if (e != cudaSuccess) return hh::note_cuda_error((int)e);
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return HH_OK;
}

// True when ptr is device (or managed) memory of device dev.
bool on_device(const void* ptr, int dev) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" int bpa_form_image_noalloc(const double* traj_xyz, int64_t n_pos, const double* freqs_hz, int32_t n_f,
                                      const hh_grid* grid, const hh_config* cfg, const void* echo_c64,
                                      void* image_c64, void* cuda_stream) {
    int st = hh::validate_inputs(traj_xyz, n_pos, freqs_hz, n_f, grid, cfg, false);
    if (st != HH_OK) return st;
    if (!echo_c64 || !image_c64) return HH_ERR_ARG;
    // Range constants and a gate covering every (voxel, position) distance,
    // derived exactly as bpa_form_image derives them.
    hh_plan tmp;
    hh::direct_bpa_setup(traj_xyz, n_pos, freqs_hz, n_f, grid, cfg, tmp);
    // Workspace layout: counters | twiddles | trajectory | range profiles.
    const size_t off_tw = align256(sizeof(int64_t) * hh::CNT_N);
    const size_t off_traj = off_tw + align256(sizeof(float2) * 2 * (size_t)tmp.n_fft);
    const size_t off_prof = off_traj + align256(sizeof(double) * 3 * (size_t)n_pos);
    const size_t need = off_prof + sizeof(float4) * (size_t)n_pos * (size_t)tmp.gate_n;
    if (need > (size_t)HH_NOALLOC_SCRATCH_BYTES) return HH_ERR_SCRATCH_LIMIT;

    void* base = nullptr;
    st = scratch_of_current_device(&base);
    if (st != HH_OK) return st;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return hh::note_cuda_error((int)e);
    if (!on_device(echo_c64, dev) || !on_device(image_c64, dev)) return HH_ERR_ARG;

    unsigned char* w = static_cast<unsigned char*>(base);
    void* d_cnt = w;
    float2* d_tw = reinterpret_cast<float2*>(w + off_tw);
    double* d_traj = reinterpret_cast<double*>(w + off_traj);
    void* d_prof = w + off_prof;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    const hh::KConst kc = hh::make_kconst(&tmp);
    // The counters accumulate atomically and must start at zero; the twiddles,
    // trajectory and every gate bin of the profiles are rewritten before use.
    // The counters are not read back (that would need a synchronisation): the gate
    // covers every voxel-position distance, so a lookup outside it cannot occur.
    e = cudaMemsetAsync(d_cnt, 0, sizeof(int64_t) * hh::CNT_N, s);
    if (e != cudaSuccess) return hh::note_cuda_error((int)e);
    e = cudaMemcpyAsync(d_traj, traj_xyz, sizeof(double) * 3 * (size_t)n_pos, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return hh::note_cuda_error((int)e);
    k_noalloc_twiddles<<<(unsigned)((2 * tmp.n_fft + 255) / 256), 256, 0, s>>>(d_tw, tmp.n_fft);
    hh::note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return hh::note_cuda_error((int)e);
    e = (cudaError_t)hh::launch_rc(echo_c64, nullptr, n_pos, n_f, tmp.n_fft, tmp.gate0, tmp.gate_n, d_tw, d_prof,
                                   nullptr, cuda_stream);
    if (e != cudaSuccess) return hh::note_cuda_error((int)e);
    e = (cudaError_t)hh::launch_bpa(d_traj, n_pos, d_prof, kc, *grid, image_c64, d_cnt, cuda_stream);
    if (e != cudaSuccess) return hh::note_cuda_error((int)e);
    return HH_OK;
}
