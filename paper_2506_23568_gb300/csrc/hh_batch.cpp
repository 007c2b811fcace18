// Batched imaging: many independent scans (uneven lengths and grids, each with its own plan)
// imaged by one CUDA graph launch.  The first call records every scan's hhffbp_form_image
// sequence into a graph, scan i on side stream i mod n_streams forked from and joined back
// to a capture stream, so that the scans run concurrently and fill the SMs together; later
// calls with the same buffers replay it with one cudaGraphLaunch.  The paper images one scan
// at a time (Sec. IV); this is the batching of many scans around its method.
#include <cuda_runtime.h>

#include <new>
#include <vector>

#include "hh_internal.h"

struct hh_batch {
    std::vector<const hh_plan*> plans;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> echo_key;
    std::vector<void*> image_key;
    int device = 0;
};

namespace {

bool device_buffer(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void release(hh_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Record the scans into a graph (any previous one is dropped).
int capture(hh_batch* b, const void* const* echos, void* const* images) {
    release(b);
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return hh::note_cuda_error((int)e);
    int st = HH_OK;
    e = cudaEventRecord(b->fork, b->cap);
    for (size_t k = 0; e == cudaSuccess && k < b->side.size(); ++k) e = cudaStreamWaitEvent(b->side[k], b->fork, 0);
    for (size_t i = 0; e == cudaSuccess && st == HH_OK && i < b->plans.size(); ++i)
        st = hhffbp_form_image(b->plans[i], echos[i], images[i], b->side[i % b->side.size()]);
    for (size_t k = 0; e == cudaSuccess && k < b->side.size(); ++k) {
        e = cudaEventRecord(b->join[k], b->side[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->join[k], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);  // always end the capture
    if (st != HH_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return hh::note_cuda_error((int)(e != cudaSuccess ? e : e2));
    }
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
        release(b);
        return hh::note_cuda_error((int)e);
    }
    b->echo_key.assign(echos, echos + b->plans.size());
    b->image_key.assign(images, images + b->plans.size());
    return HH_OK;
}

}  // namespace

extern "C" {

int hhffbp_batch_create(hh_plan* const* plans, int32_t n_plans, int32_t n_streams, hh_batch** out) {
    if (!out) return HH_ERR_ARG;
    *out = nullptr;
    if (!plans || n_plans <= 0 || n_streams <= 0) return HH_ERR_ARG;
    for (int32_t i = 0; i < n_plans; ++i) {
        if (!plans[i]) return HH_ERR_ARG;
        if (!plans[i]->on_device) return HH_ERR_HOST_ONLY;
    }
    hh_batch* b = new (std::nothrow) hh_batch();
    if (!b) return HH_ERR_OOM;
    b->plans.assign(plans, plans + n_plans);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    const int ns = n_streams < n_plans ? n_streams : n_plans;
    for (int k = 0; e == cudaSuccess && k < ns; ++k) {
        cudaStream_t s = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->side.push_back(s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->join.push_back(ev);
    }
    if (e != cudaSuccess) {
        hhffbp_batch_destroy(b);
        return hh::note_cuda_error((int)e);
    }
    *out = b;
    return HH_OK;
}

int hhffbp_batch_form_images(hh_batch* b, const void* const* echos, void* const* images, void* cuda_stream) {
    if (!b || !echos || !images) return HH_ERR_ARG;
    const size_t n = b->plans.size();
    for (size_t i = 0; i < n; ++i)
        if (!echos[i] || !images[i] || !device_buffer(echos[i]) || !device_buffer(images[i])) return HH_ERR_ARG;
    bool same = b->exec != nullptr;
    for (size_t i = 0; same && i < n; ++i) same = echos[i] == b->echo_key[i] && images[i] == b->image_key[i];
    if (!same) {
        if (int st = capture(b, echos, images)) return st;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return hh::note_cuda_error((int)e);
    for (const hh_plan* p : b->plans) const_cast<hh_plan*>(p)->last_stream = cuda_stream;
    return HH_OK;
}

int hhffbp_batch_destroy(hh_batch* b) {
    if (!b) return HH_OK;
    if (b->cap) cudaStreamSynchronize(b->cap);
    release(b);
    for (cudaStream_t s : b->side) cudaStreamDestroy(s);
    for (cudaEvent_t ev : b->join) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return HH_OK;
}

}  // extern "C"
