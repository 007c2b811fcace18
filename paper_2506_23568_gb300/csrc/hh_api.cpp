// C ABI of the HHFFBPA library: argument checks, device workspace, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <unordered_map>

#include "hh_internal.h"

namespace {

thread_local int g_last_cuda = 0;

int fail_cuda(cudaError_t e) {
    g_last_cuda = (int)e;
    return e == cudaErrorMemoryAllocation ? HH_ERR_OOM : HH_ERR_CUDA;
}

#define HH_CUDA(call)                              \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return fail_cuda(e_); \
    } while (0)

#define HH_LAUNCH(call)                                        \
    do {                                                       \
        int e_ = (call);                                       \
        if (e_ != 0) return fail_cuda((cudaError_t)e_);        \
    } while (0)

// true when ptr is host memory (pageable or page-locked), false for device/managed memory
bool is_host_pointer(const void* ptr) {
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear: unregistered host pointers report an error on some drivers
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

// Per-device cache of device blocks released by destroyed plans, so that the
// per-scan plan of a repeated workload does not pay cudaMalloc/cudaFree.
// Sizes are rounded up to 2 MiB; a request takes the smallest cached block of
// at least its size and at most twice it.  hh_release_cached_memory() frees all.
struct BlockCache {
    std::mutex mu;
    std::multimap<std::pair<int, size_t>, void*> free_blocks;  // (device, bytes) -> block
    std::unordered_map<void*, std::pair<int, size_t>> sizes;   // every live or cached block
    size_t cached_bytes = 0;
    static constexpr size_t kCap = (size_t)64 << 30;
};
BlockCache& cache() {
    static BlockCache* c = new BlockCache();  // never destroyed: safe at process exit
    return *c;
}

size_t round_block(size_t bytes) {
    const size_t g = (size_t)2 << 20;
    return bytes <= ((size_t)1 << 20) ? ((bytes + 255) & ~(size_t)255) : (bytes + g - 1) / g * g;
}

cudaError_t cached_malloc(void** ptr, size_t bytes, int device) {
    BlockCache& c = cache();
    const size_t want = round_block(bytes);
    {
        std::lock_guard<std::mutex> lk(c.mu);
        auto it = c.free_blocks.lower_bound({device, want});
        if (it != c.free_blocks.end() && it->first.first == device && it->first.second <= 2 * want) {
            *ptr = it->second;
            c.cached_bytes -= it->first.second;
            c.free_blocks.erase(it);
            return cudaSuccess;
        }
    }
    cudaError_t e = cudaMalloc(ptr, want);
    if (e == cudaErrorMemoryAllocation) {  // return this device's cached blocks and retry once
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(c.mu);
        for (auto it = c.free_blocks.begin(); it != c.free_blocks.end();) {
            if (it->first.first == device) {
                cudaFree(it->second);
                c.sizes.erase(it->second);
                c.cached_bytes -= it->first.second;
                it = c.free_blocks.erase(it);
            } else {
                ++it;
            }
        }
        e = cudaMalloc(ptr, want);
    }
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(c.mu);
        c.sizes[*ptr] = {device, want};
    }
    return e;
}

void cached_free(void* ptr) {
    BlockCache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.sizes.find(ptr);
    if (it == c.sizes.end()) {
        cudaFree(ptr);
        return;
    }
    if (c.cached_bytes + it->second.second > BlockCache::kCap) {
        cudaFree(ptr);
        c.sizes.erase(it);
        return;
    }
    c.free_blocks.insert({it->second, ptr});
    c.cached_bytes += it->second.second;
}

int dev_alloc(hh_plan* p, void** ptr, size_t bytes) {
    if (bytes == 0) bytes = 16;
    HH_CUDA(cached_malloc(ptr, bytes, p->device));
    p->workspace_bytes += (int64_t)bytes;
    return HH_OK;
}

void free_device(hh_plan* p) {
    void** bufs[] = {&p->d_tile_off, &p->d_nodes, &p->d_mem_pos, &p->d_perm, &p->d_prof, &p->d_pool[0], &p->d_pool[1],
                     &p->d_twiddle, &p->d_counters, &p->d_echo_stage, &p->d_image_stage,
                     &p->d_need, &p->d_xyz, &p->d_nodev, &p->d_tile_ref, &p->d_tiles, &p->d_pair_off, &p->d_pairs, &p->d_prof2,
                     &p->d_fb_segs, &p->d_fb_recs, &p->d_fb_vals, &p->d_fb_fixes, &p->d_fb_counts};
    for (void** b : bufs)
        if (*b) {
            cached_free(*b);
            *b = nullptr;
        }
    for (void*& ev : p->events)
        if (ev) {
            cudaEventDestroy(static_cast<cudaEvent_t>(ev));
            ev = nullptr;
        }
}

// Stage profiling: event i marks the start of stage i (and the end of stage i - 1).
struct StageMarks {
    hh_plan* p;
    cudaStream_t s;
    int n = 0;
    int mark(int kind, int level) {
        if (!p->profile) return HH_OK;
        if ((int)p->events.size() <= n) {
            cudaEvent_t ev;
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return fail_cuda(e);
            p->events.push_back(ev);
        }
        cudaError_t e = cudaEventRecord(static_cast<cudaEvent_t>(p->events[n]), s);
        if (e != cudaSuccess) return fail_cuda(e);
        if (kind >= 0) {
            p->stage_kind.push_back(kind);
            p->stage_level.push_back(level);
        }
        ++n;
        return HH_OK;
    }
};

std::vector<hh::DNode> device_nodes(const hh_plan* p) {
    std::vector<hh::DNode> out(p->nodes.size());
    for (size_t i = 0; i < p->nodes.size(); ++i) {
        const hh::HNode& h = p->nodes[i];
        hh::DNode d{};
        const double a = h.rect[0], b = h.rect[1], e = h.rect[2], g = h.rect[3];
        d.cx = 0.5 * (a + b);
        d.cy = 0.5 * (e + g);
        d.cz = h.zbar;
        d.hxd = 0.5 * (b - a);
        d.hyd = 0.5 * (g - e);
        d.hx = (float)d.hxd;
        d.hy = (float)d.hyd;
        d.C2 = (float)(4 * (b - a) * (b - a) + 4 * (g - e) * (g - e));
        d.usat = (float)(p->kmax / hh::kPi * (b - a));
        d.vsat = (float)(p->kmax / hh::kPi * (g - e));
        for (int k = 0; k < 3; ++k) {
            d.lo[k] = (float)h.lo[k];
            d.eta[k] = (float)h.eta[k];
            d.N[k] = (int32_t)h.N[k];
        }
        d.mem_begin = (int32_t)h.begin;
        d.mem_end = (int32_t)h.end;
        d.child0 = (int32_t)h.child0;
        d.nchild = (int32_t)h.nchild;
        d.pool_off = h.pool_off;
        out[i] = d;
    }
    return out;
}

// Member positions in tree order (FP64) and, per non-root level, each member relative to the
// centre of its node: v = centre - p' and |v|^2 / 2 (FP32), level-major.
// Entries of the two member arrays: positions in tree order (3 doubles each) and, per level
// below the root, every member relative to its node's centre with |v|^2 / 2 (4 floats).
size_t n_mem_pos(const hh_plan* p) { return 3 * (size_t)p->n_pos; }
size_t n_nodev(const hh_plan* p) { return 4 * (size_t)p->n_pos * (size_t)std::max(1, p->n_levels - 1); }

// Process-wide host staging of the member arrays, reused by every plan (no zero fill and no
// fresh pages per plan).  A cudaMemcpyAsync from pageable memory returns once its source has
// been copied out, so the buffers are free again after the uploads; the mutex serialises
// their users.
struct MemberStage {
    std::mutex mu;
    std::unique_ptr<double[]> pos;
    std::unique_ptr<float[]> vec;
    size_t pos_cap = 0, vec_cap = 0;
};
MemberStage& member_stage() {
    static MemberStage m;
    return m;
}

// Fills mem_pos [n_mem_pos] and nodev [n_nodev] (every entry).
void member_arrays(const hh_plan* p, const std::vector<hh::DNode>& dn, double* mem_pos, float* nodev) {
    const int64_t n_pos = p->n_pos;
    const int64_t blk = 4096;  // positions in tree order, gathered in blocks
    hh::parallel_for((n_pos + blk - 1) / blk, n_pos >= 32768 ? 16 : 1, [&](int64_t b) {
        for (int64_t q = b * blk; q < std::min(n_pos, (b + 1) * blk); ++q)
            for (int k = 0; k < 3; ++k) mem_pos[3 * q + k] = p->traj[3 * p->perm[q] + k];
    });
    if (p->n_levels < 2) std::fill(nodev, nodev + n_nodev(p), 0.f);  // no level below a root leaf
    const int64_t n_vec_nodes = p->n_levels > 1 ? p->level_start[p->n_levels - 1] : 0;
    hh::parallel_for(n_vec_nodes, n_pos >= 32768 ? 16 : 1, [&](int64_t j) {  // nodes of levels 0 .. L-2
        float* out_l = nodev + 4 * (size_t)n_pos * (size_t)p->nodes[j].level;
        const hh::DNode& L = dn[j];
        for (int64_t q = L.mem_begin; q < L.mem_end; ++q) {
            const float vx = (float)(L.cx - mem_pos[3 * q]), vy = (float)(L.cy - mem_pos[3 * q + 1]),
                        vz = (float)(L.cz - mem_pos[3 * q + 2]);
            out_l[4 * q] = vx;
            out_l[4 * q + 1] = vy;
            out_l[4 * q + 2] = vz;
            out_l[4 * q + 3] = 0.5f * std::fmaf(vx, vx, std::fmaf(vy, vy, vz * vz));
        }
    });
}

int upload(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    HH_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
    return HH_OK;
}

// Member arrays of plan p, computed into the shared staging buffers and copied to the plan's
// device arrays on stream s.
int upload_member_arrays(const hh_plan* p, const std::vector<hh::DNode>& dn, cudaStream_t s) {
    MemberStage& ms = member_stage();
    std::lock_guard<std::mutex> lk(ms.mu);
    const size_t np = n_mem_pos(p), nv = n_nodev(p);
    if (ms.pos_cap < np) {
        ms.pos.reset(new (std::nothrow) double[np]);
        ms.pos_cap = ms.pos ? np : 0;
    }
    if (ms.vec_cap < nv) {
        ms.vec.reset(new (std::nothrow) float[nv]);
        ms.vec_cap = ms.vec ? nv : 0;
    }
    if (!ms.pos || !ms.vec) return HH_ERR_OOM;
    member_arrays(p, dn, ms.pos.get(), ms.vec.get());
    if (int r = upload(p->d_mem_pos, ms.pos.get(), sizeof(double) * np, s)) return r;
    return upload(p->d_nodev, ms.vec.get(), sizeof(float) * nv, s);
}

#define HH_TRY(expr)            \
    do {                        \
        int r_ = (expr);        \
        if (r_ != HH_OK) {      \
            free_device(p);     \
            delete p;           \
            return r_;          \
        }                       \
    } while (0)

}  // namespace

namespace hh {
int note_cuda_error(int cuda_error) { return fail_cuda((cudaError_t)cuda_error); }

// Kernel launches issued by the library since the process started (every launch site calls it).
static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace hh

extern "C" {

int hhffbp_default_config(hh_config* cfg) {
    if (!cfg) return HH_ERR_ARG;
    cfg->leaf_size = 32;
    cfg->merge_factor = 4;
    cfg->eta = 2.0f;
    cfg->taps = 6;
    cfg->range_os = 16;
    cfg->flags = 0;
    return HH_OK;
}

int hhffbp_interp_weights(int32_t taps, double eta, const double* tau, int64_t n, double* out) {
    if ((taps != 4 && taps != 6) || !(eta >= 1.0) || n < 0 || (n > 0 && (!tau || !out))) return HH_ERR_ARG;
    const hh::WPoly wp = hh::weight_poly(taps, eta);
    for (int64_t i = 0; i < n; ++i) {  // the kernels' evaluation (footprint()), in FP32 with fused multiply-adds
        const float x = std::fmaf(2.f, (float)tau[i], -1.f), x2 = x * x;
        for (int q = 0; q < taps / 2; ++q) {
            float e = wp.e[q][4], o = wp.o[q][3];
            for (int j = 3; j >= 0; --j) e = std::fmaf(e, x2, wp.e[q][j]);
            for (int j = 2; j >= 0; --j) o = std::fmaf(o, x2, wp.o[q][j]);
            out[i * taps + q] = std::fmaf(x, o, e);
            out[i * taps + taps - 1 - q] = std::fmaf(-x, o, e);
        }
    }
    return HH_OK;
}

int hhffbp_plan(const double* traj_xyz, int64_t n_pos, const double* freqs_hz, int32_t n_f, const hh_grid* grid,
                const hh_config* cfg, void* cuda_stream, hh_plan** out) {
    if (!out) return HH_ERR_ARG;
    *out = nullptr;
    int st = hh::validate_inputs(traj_xyz, n_pos, freqs_hz, n_f, grid, cfg, true);
    if (st != HH_OK) return st;
    hh_plan* p = new (std::nothrow) hh_plan();
    if (!p) return HH_ERR_OOM;
    p->n_pos = n_pos;
    p->n_f = n_f;
    p->grid = *grid;
    p->cfg = *cfg;
    p->traj.assign(traj_xyz, traj_xyz + 3 * n_pos);
    p->freqs.assign(freqs_hz, freqs_hz + n_f);
    HH_TRY(hh::build_host_plan(p));
    for (const auto& nd : p->nodes)
        for (int k = 0; k < 3; ++k)
            if (nd.N[k] > INT32_MAX / 4) {
                delete p;
                return HH_ERR_ARG;
            }
    if (cfg->flags & HH_FLAG_HOST_ONLY) {
        *out = p;
        return HH_OK;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        g_last_cuda = (int)cudaGetLastError();
        delete p;
        return HH_ERR_CUDA;
    }
    std::vector<hh::DNode> dn = device_nodes(p);
    std::vector<float> tw = hh::twiddle_table(p->n_fft);
    const int64_t n_vox = (int64_t)grid->nx * grid->ny * grid->nz;
    HH_TRY(dev_alloc(p, &p->d_nodes, sizeof(hh::DNode) * dn.size()));
    HH_TRY(dev_alloc(p, &p->d_tile_off, sizeof(int64_t) * p->tile_off.size()));
    HH_TRY(dev_alloc(p, &p->d_mem_pos, sizeof(double) * n_mem_pos(p)));
    HH_TRY(dev_alloc(p, &p->d_perm, sizeof(int64_t) * n_pos));
    HH_TRY(dev_alloc(p, &p->d_nodev, sizeof(float) * n_nodev(p)));
    HH_TRY(dev_alloc(p, &p->d_prof, 16 * (size_t)n_pos * (size_t)p->gate_n));
    HH_TRY(dev_alloc(p, &p->d_prof2, 8 * (size_t)n_pos * (size_t)((p->gate_n + 2) & ~(int64_t)1)));
    if (p->max_pool > 0) {
        HH_TRY(dev_alloc(p, &p->d_pool[0], 8 * (size_t)p->max_pool));
        HH_TRY(dev_alloc(p, &p->d_pool[1], 8 * (size_t)p->max_pool));
    }
    if (p->n_levels > 1) {  // tile warm starts of the lattice levels
        p->tile_ref_base.assign(p->n_levels, 0);
        int64_t tiles = 0;
        for (int l = 0; l + 1 < p->n_levels; ++l) {
            p->tile_ref_base[l] = tiles;
            tiles += p->level_tiles[l];
        }
        if (tiles > 0) HH_TRY(dev_alloc(p, &p->d_tile_ref, sizeof(float) * 16 * (size_t)tiles));
        if (tiles > 0) HH_TRY(dev_alloc(p, &p->d_tiles, sizeof(hh::DTile) * (size_t)tiles));
        p->pair_base.assign(p->n_levels, 0);
        int64_t pairs = 0;
        for (int l = 0; l + 1 < p->n_levels; ++l) {
            p->pair_base[l] = pairs;
            pairs += p->level_pairs[l];
        }
        if (pairs > 0) {
            HH_TRY(dev_alloc(p, &p->d_pairs, 8 * (size_t)pairs));
            HH_TRY(dev_alloc(p, &p->d_pair_off, sizeof(int64_t) * p->pair_off.size()));
        }
    }
    if (p->n_levels > 1) {  // deferred-fallback queue, sized for the widest merge level
        int64_t segs = 1, widest = 1;
        for (int l = 1; l < p->n_levels; ++l) {
            const int64_t nch = p->nodes[p->level_start[l]].nchild;
            segs = std::max(segs, p->level_tiles[l] * nch);
            widest = std::max(widest, p->level_samples[l] * nch);
        }
        p->fb_seg_cap = segs;  // at most one segment per (tile, child): never full
        p->fb_rec_cap = std::min<int64_t>(std::max<int64_t>(widest / 4, 1 << 16), (int64_t)1 << 25);
        HH_TRY(dev_alloc(p, &p->d_fb_segs, sizeof(hh::FbSeg) * (size_t)p->fb_seg_cap));
        HH_TRY(dev_alloc(p, &p->d_fb_recs, sizeof(hh::FbRec) * (size_t)p->fb_rec_cap));
        HH_TRY(dev_alloc(p, &p->d_fb_vals, 8 * (size_t)p->fb_rec_cap));
        HH_TRY(dev_alloc(p, &p->d_fb_fixes, sizeof(hh::FbFix) * (size_t)p->fb_rec_cap));
        HH_TRY(dev_alloc(p, &p->d_fb_counts, 32));
    }
    if (p->need_total > 0) HH_TRY(dev_alloc(p, &p->d_need, sizeof(uint32_t) * (size_t)p->need_total));
    if (p->xyz_total > 0) HH_TRY(dev_alloc(p, &p->d_xyz, 16 * (size_t)p->xyz_total));
    HH_TRY(dev_alloc(p, &p->d_twiddle, sizeof(float) * tw.size()));
    HH_TRY(dev_alloc(p, &p->d_counters, sizeof(int64_t) * hh::CNT_N));
    HH_TRY(dev_alloc(p, &p->d_echo_stage, 8 * (size_t)n_pos * (size_t)n_f));
    HH_TRY(dev_alloc(p, &p->d_image_stage, 8 * (size_t)n_vox));
    HH_TRY(upload(p->d_nodes, dn.data(), sizeof(hh::DNode) * dn.size(), s));
    if (!p->tile_off.empty())
        HH_TRY(upload(p->d_tile_off, p->tile_off.data(), sizeof(int64_t) * p->tile_off.size(), s));
    if (p->d_pair_off)
        HH_TRY(upload(p->d_pair_off, p->pair_off.data(), sizeof(int64_t) * p->pair_off.size(), s));
    HH_TRY(upload_member_arrays(p, dn, s));
    HH_TRY(upload(p->d_perm, p->perm.data(), sizeof(int64_t) * n_pos, s));
    HH_TRY(upload(p->d_twiddle, tw.data(), sizeof(float) * tw.size(), s));
    if (p->d_tiles) {
        const int te = hh::launch_tile_table(p, cuda_stream);
        if (te != 0) {
            free_device(p);
            delete p;
            return fail_cuda((cudaError_t)te);
        }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        free_device(p);
        delete p;
        return fail_cuda(e);
    }
    p->on_device = true;
    p->last_stream = cuda_stream;
    *out = p;
    return HH_OK;
}

int hhffbp_plan_update_positions(hh_plan* p, const double* traj_xyz, void* cuda_stream) {
    if (!p || !traj_xyz) return HH_ERR_ARG;
    for (int64_t q = 0; q < 3 * p->n_pos; ++q)
        if (!std::isfinite(traj_xyz[q])) return HH_ERR_ARG;
    p->traj.assign(traj_xyz, traj_xyz + 3 * p->n_pos);
    if (!p->on_device) return HH_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    if (int r = upload_member_arrays(p, device_nodes(p), s)) return r;
    HH_CUDA(cudaStreamSynchronize(s));  // the new positions are in place on return
    p->last_stream = cuda_stream;
    return HH_OK;
}

int hhffbp_plan_destroy(hh_plan* plan) {
    if (!plan) return HH_OK;
    if (plan->on_device) {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != plan->device) cudaSetDevice(plan->device);
        cudaDeviceSynchronize();
        free_device(plan);
        if (cur != plan->device) cudaSetDevice(cur);
    }
    delete plan;
    return HH_OK;
}

int hhffbp_plan_info(const hh_plan* p, hh_plan_info* info) {
    if (!p || !info) return HH_ERR_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n_levels = p->n_levels;
    info->depth_leaves = p->depth_leaves;
    info->n_nodes = (int64_t)p->nodes.size();
    for (int l = 0; l < p->n_levels && l < 32; ++l) {
        info->level_nodes[l] = p->level_start[l + 1] - p->level_start[l];
        info->level_samples[l] = p->level_samples[l];
    }
    info->workspace_bytes = p->workspace_bytes;
    info->n_fft = p->n_fft;
    info->gate_start = p->gate0;
    info->gate_bins = p->gate_n;
    info->dR = p->dR;
    info->kc = p->kc;
    return HH_OK;
}

int hhffbp_plan_export(const hh_plan* p, int64_t* perm, int64_t* nodes_i, double* nodes_d, double* scalars) {
    if (!p) return HH_ERR_ARG;
    if (scalars) {
        scalars[0] = p->zbar_all;
        scalars[1] = p->kmin;
        scalars[2] = p->kmax;
        scalars[3] = p->zh_floor;
        scalars[4] = p->grid.z0 + 0.5 * p->grid.dz * (p->grid.nz - 1) - p->zbar_all;
    }
    if (perm) std::memcpy(perm, p->perm.data(), sizeof(int64_t) * p->perm.size());
    for (size_t k = 0; k < p->nodes.size(); ++k) {
        const hh::HNode& n = p->nodes[k];
        if (nodes_i) {
            int64_t* I = nodes_i + 10 * k;
            I[0] = n.level; I[1] = n.depth; I[2] = n.t; I[3] = n.begin; I[4] = n.end;
            I[5] = n.child0; I[6] = n.nchild; I[7] = n.N[0]; I[8] = n.N[1]; I[9] = n.N[2];
        }
        if (nodes_d) {
            double* F = nodes_d + 11 * k;
            for (int q = 0; q < 4; ++q) F[q] = n.rect[q];
            for (int q = 0; q < 3; ++q) F[4 + q] = n.lo[q];
            for (int q = 0; q < 3; ++q) F[7 + q] = n.eta[q];
            F[10] = n.zbar;
        }
    }
    return HH_OK;
}

int hhffbp_form_image(const hh_plan* cp, const void* echo_c64, void* image_c64, void* cuda_stream) {
    if (!cp || !echo_c64 || !image_c64) return HH_ERR_ARG;
    if (!cp->on_device) return HH_ERR_HOST_ONLY;
    hh_plan* p = const_cast<hh_plan*>(cp);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    const int64_t n_vox = (int64_t)p->grid.nx * p->grid.ny * p->grid.nz;
    const bool host_echo = is_host_pointer(echo_c64), host_img = is_host_pointer(image_c64);
    const void* echo = echo_c64;
    void* image = image_c64;
    StageMarks sm{p, s};
    p->stage_kind.clear();
    p->stage_level.clear();
#define HH_MARK(kind, level)                  \
    do {                                      \
        int r_ = sm.mark((kind), (level));    \
        if (r_ != HH_OK) return r_;           \
    } while (0)
    if (host_echo) {
        HH_MARK(HH_STAGE_H2D, -1);
        HH_CUDA(cudaMemcpyAsync(p->d_echo_stage, echo_c64, 8 * (size_t)p->n_pos * p->n_f, cudaMemcpyHostToDevice, s));
        echo = p->d_echo_stage;
    }
    if (host_img) image = p->d_image_stage;
    HH_MARK(HH_STAGE_RC, -1);
    HH_CUDA(cudaMemsetAsync(p->d_counters, 0, sizeof(int64_t) * hh::CNT_N, s));
    const hh::KConst kc = hh::make_kconst(p);
    // the factorised forward reads P-only rows (windows, fallbacks); the (P, dP) pair rows serve
    // a single-level plan's direct BPA and the gradient
    HH_LAUNCH(hh::launch_rc(echo, static_cast<const int64_t*>(p->d_perm), p->n_pos, p->n_f, p->n_fft, p->gate0,
                            p->gate_n, p->d_twiddle, p->n_levels == 1 ? p->d_prof : nullptr, p->d_prof2,
                            cuda_stream));
    if (p->n_levels > 1) {
        // top-down: which lattice samples the image needs (the footprints of needed points)
        HH_MARK(HH_STAGE_NEED_FINAL, p->n_levels - 1);
        for (int l = 0; l + 1 < p->n_levels; ++l) HH_LAUNCH(hh::launch_tile_refs(p, kc, l, cuda_stream));
        HH_CUDA(cudaMemsetAsync(p->d_need, 0, sizeof(uint32_t) * (size_t)p->need_total, s));
        HH_LAUNCH(hh::launch_need_final(p, kc, cuda_stream));
        for (int l = p->n_levels - 2; l >= 1; --l) {
            HH_MARK(HH_STAGE_NEED_LEVEL, l);
            HH_LAUNCH(hh::launch_need_level(p, kc, l, cuda_stream));
        }
        // bottom-up: values at the needed samples
        HH_MARK(HH_STAGE_LEAF, 0);
        HH_LAUNCH(hh::launch_stage0(p, kc, cuda_stream));
        for (int l = 1; l + 1 < p->n_levels; ++l) {
            HH_MARK(HH_STAGE_MERGE, l);
            HH_CUDA(cudaMemsetAsync(p->d_fb_counts, 0, 32, s));
            HH_LAUNCH(hh::launch_merge(p, kc, l, cuda_stream));
            HH_LAUNCH(hh::launch_deferred(p, kc, l, p->d_pool[l & 1], cuda_stream));
        }
    }
    HH_MARK(HH_STAGE_FINAL, p->n_levels - 1);
    if (p->n_levels > 1) HH_CUDA(cudaMemsetAsync(p->d_fb_counts, 0, 32, s));
    HH_LAUNCH(hh::launch_final(p, kc, image, cuda_stream));
    if (p->n_levels > 1) HH_LAUNCH(hh::launch_deferred(p, kc, p->n_levels - 1, image, cuda_stream));
    if (host_img) {
        HH_MARK(HH_STAGE_D2H, -1);
        HH_CUDA(cudaMemcpyAsync(image_c64, image, 8 * (size_t)n_vox, cudaMemcpyDeviceToHost, s));
    }
    HH_MARK(-1, -1);
#undef HH_MARK
    p->last_stream = cuda_stream;
    return HH_OK;
}

int hhffbp_plan_profile(hh_plan* p, int enable) {
    if (!p) return HH_ERR_ARG;
    if (!p->on_device) return HH_ERR_HOST_ONLY;
    p->profile = enable != 0;
    return HH_OK;
}

int hhffbp_plan_stage_times(const hh_plan* p, float* ms, int32_t* kind, int32_t* level, int32_t max_n,
                            int32_t* n_out) {
    if (!p || !n_out || max_n < 0) return HH_ERR_ARG;
    *n_out = 0;
    if (!p->on_device) return HH_ERR_HOST_ONLY;
    const int n = (int)p->stage_kind.size();
    if (n == 0) return HH_OK;
    HH_CUDA(cudaEventSynchronize(static_cast<cudaEvent_t>(p->events[n])));
    const int m = n < max_n ? n : max_n;
    for (int i = 0; i < m; ++i) {
        if (ms) {
            float t = 0.f;
            HH_CUDA(cudaEventElapsedTime(&t, static_cast<cudaEvent_t>(p->events[i]),
                                         static_cast<cudaEvent_t>(p->events[i + 1])));
            ms[i] = t;
        }
        if (kind) kind[i] = p->stage_kind[i];
        if (level) level[i] = p->stage_level[i];
    }
    *n_out = m;
    return HH_OK;
}

int hhffbp_plan_counters(const hh_plan* p, int64_t out[8]) {
    if (!p || !out) return HH_ERR_ARG;
    std::memset(out, 0, sizeof(int64_t) * 8);
    if (!p->on_device) return HH_ERR_HOST_ONLY;
    int64_t all[hh::CNT_N];
    cudaStream_t s = reinterpret_cast<cudaStream_t>(p->last_stream);
    HH_CUDA(cudaStreamSynchronize(s));
    HH_CUDA(cudaMemcpy(all, p->d_counters, sizeof(int64_t) * hh::CNT_N, cudaMemcpyDeviceToHost));
    std::memcpy(out, all, sizeof(int64_t) * 8);
    if (out[hh::CNT_GATE_MISS] != 0 || out[hh::CNT_ERROR] != 0) return HH_ERR_DEVICE_FLAG;
    return HH_OK;
}

int hhffbp_plan_level_counts(const hh_plan* p, int64_t* evaluated, int32_t max_levels) {
    if (!p || !evaluated || max_levels < 0) return HH_ERR_ARG;
    if (!p->on_device) return HH_ERR_HOST_ONLY;
    int64_t all[hh::CNT_N];
    HH_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(p->last_stream)));
    HH_CUDA(cudaMemcpy(all, p->d_counters, sizeof(int64_t) * hh::CNT_N, cudaMemcpyDeviceToHost));
    for (int l = 0; l < max_levels && l < p->n_levels; ++l)
        evaluated[l] = (l == p->n_levels - 1) ? p->level_samples[l] : all[hh::CNT_NEEDED + l];
    return HH_OK;
}

}  // extern "C"

namespace hh {
// Range constants and a gate of stored bins covering every (voxel, position)
// distance: the setup of direct BPA, its gradient, its adjoint and the
// fixed-workspace variant.
void direct_bpa_setup(const double* traj_xyz, int64_t n_pos, const double* freqs_hz, int32_t n_f, const hh_grid* grid,
                      const hh_config* cfg, hh_plan& tmp) {
    tmp.n_pos = n_pos;
    tmp.n_f = n_f;
    tmp.grid = *grid;
    tmp.cfg = *cfg;
    hh::range_constants(freqs_hz, n_f, cfg->range_os, &tmp.kmin, &tmp.kmax, &tmp.kc, &tmp.dk, &tmp.n_fft, &tmp.dR);
    double smin = 0, smax = 0;
    const double lo[3] = {grid->x0, grid->y0, grid->z0};
    const double hi[3] = {grid->x0 + grid->dx * (grid->nx - 1), grid->y0 + grid->dy * (grid->ny - 1),
                          grid->z0 + grid->dz * (grid->nz - 1)};
    for (int i = 0; i < 3; ++i) {
        double tl = HUGE_VAL, th = -HUGE_VAL;
        for (int64_t q = 0; q < n_pos; ++q) {
            tl = std::fmin(tl, traj_xyz[3 * q + i]);
            th = std::fmax(th, traj_xyz[3 * q + i]);
        }
        const double gap = std::fmax(0.0, std::fmax(lo[i] - th, tl - hi[i]));
        const double span = std::fmax(std::fabs(hi[i] - tl), std::fabs(th - lo[i]));
        smin += gap * gap;
        smax += span * span;
    }
    tmp.gate0 = (int64_t)std::floor(std::sqrt(smin) / tmp.dR) - 2;
    tmp.gate_n = (int64_t)std::ceil(std::sqrt(smax) / tmp.dR) + 3 - tmp.gate0;
    tmp.gate_wrap = false;
    if (tmp.gate_n >= tmp.n_fft) {
        tmp.gate0 = 0;
        tmp.gate_n = tmp.n_fft;
        tmp.gate_wrap = true;
    }
}
}  // namespace hh

extern "C" {

int bpa_form_image(const double* traj_xyz, int64_t n_pos, const double* freqs_hz, int32_t n_f, const hh_grid* grid,
                   const hh_config* cfg, const void* echo_c64, void* image_c64, void* cuda_stream) {
    int st = hh::validate_inputs(traj_xyz, n_pos, freqs_hz, n_f, grid, cfg, false);
    if (st != HH_OK) return st;
    if (!echo_c64 || !image_c64) return HH_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    hh_plan tmp;
    hh::direct_bpa_setup(traj_xyz, n_pos, freqs_hz, n_f, grid, cfg, tmp);
    const hh::KConst kc = hh::make_kconst(&tmp);
    std::vector<float> tw = hh::twiddle_table(tmp.n_fft);
    const int64_t n_vox = (int64_t)grid->nx * grid->ny * grid->nz;
    const bool host_echo = is_host_pointer(echo_c64), host_img = is_host_pointer(image_c64);
    void *d_traj = nullptr, *d_prof = nullptr, *d_tw = nullptr, *d_cnt = nullptr, *d_echo = nullptr, *d_img = nullptr;
    auto release = [&]() {
        for (void* b : {d_traj, d_prof, d_tw, d_cnt, d_echo, d_img})
            if (b) cudaFreeAsync(b, s);
    };
#define HH_STEP(call)                          \
    do {                                       \
        cudaError_t e_ = (cudaError_t)(call);  \
        if (e_ != cudaSuccess) {               \
            release();                         \
            return fail_cuda(e_);              \
        }                                      \
    } while (0)
    HH_STEP(cudaMallocAsync(&d_traj, sizeof(double) * 3 * n_pos, s));
    HH_STEP(cudaMallocAsync(&d_prof, 16 * (size_t)n_pos * (size_t)tmp.gate_n, s));
    HH_STEP(cudaMallocAsync(&d_tw, sizeof(float) * tw.size(), s));
    HH_STEP(cudaMallocAsync(&d_cnt, sizeof(int64_t) * hh::CNT_N, s));
    const void* echo = echo_c64;
    void* image = image_c64;
    if (host_echo) {
        HH_STEP(cudaMallocAsync(&d_echo, 8 * (size_t)n_pos * n_f, s));
        HH_STEP(cudaMemcpyAsync(d_echo, echo_c64, 8 * (size_t)n_pos * n_f, cudaMemcpyHostToDevice, s));
        echo = d_echo;
    }
    if (host_img) {
        HH_STEP(cudaMallocAsync(&d_img, 8 * (size_t)n_vox, s));
        image = d_img;
    }
    HH_STEP(cudaMemcpyAsync(d_traj, traj_xyz, sizeof(double) * 3 * n_pos, cudaMemcpyHostToDevice, s));
    HH_STEP(cudaMemcpyAsync(d_tw, tw.data(), sizeof(float) * tw.size(), cudaMemcpyHostToDevice, s));
    HH_STEP(cudaMemsetAsync(d_cnt, 0, sizeof(int64_t) * hh::CNT_N, s));
    HH_STEP(hh::launch_rc(echo, nullptr, n_pos, n_f, tmp.n_fft, tmp.gate0, tmp.gate_n, d_tw, d_prof, nullptr,
                          cuda_stream));
    HH_STEP(hh::launch_bpa(static_cast<const double*>(d_traj), n_pos, d_prof, kc, *grid, image, d_cnt, cuda_stream));
    if (host_img) HH_STEP(cudaMemcpyAsync(image_c64, image, 8 * (size_t)n_vox, cudaMemcpyDeviceToHost, s));
    release();
#undef HH_STEP
    return HH_OK;
}

int bpa_traj_gradient(const double* traj_xyz, int64_t n_pos, const double* freqs_hz, int32_t n_f,
                      const hh_grid* grid, const hh_config* cfg, const void* echo_c64, const void* grad_image_c64,
                      double* grad_traj, void* cuda_stream) {
    int st = hh::validate_inputs(traj_xyz, n_pos, freqs_hz, n_f, grid, cfg, false);
    if (st != HH_OK) return st;
    if (!echo_c64 || !grad_image_c64 || !grad_traj) return HH_ERR_ARG;
    if (is_host_pointer(grad_image_c64) || is_host_pointer(grad_traj)) return HH_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    hh_plan tmp;
    hh::direct_bpa_setup(traj_xyz, n_pos, freqs_hz, n_f, grid, cfg, tmp);
    const hh::KConst kc = hh::make_kconst(&tmp);
    std::vector<float> tw = hh::twiddle_table(tmp.n_fft);
    const bool host_echo = is_host_pointer(echo_c64);
    void *d_traj = nullptr, *d_prof = nullptr, *d_tw = nullptr, *d_cnt = nullptr, *d_echo = nullptr;
    auto release = [&]() {
        for (void* b : {d_traj, d_prof, d_tw, d_cnt, d_echo})
            if (b) cudaFreeAsync(b, s);
    };
#define HH_STEP(call)                          \
    do {                                       \
        cudaError_t e_ = (cudaError_t)(call);  \
        if (e_ != cudaSuccess) {               \
            release();                         \
            return fail_cuda(e_);              \
        }                                      \
    } while (0)
    HH_STEP(cudaMallocAsync(&d_traj, sizeof(double) * 3 * n_pos, s));
    HH_STEP(cudaMallocAsync(&d_prof, 16 * (size_t)n_pos * (size_t)tmp.gate_n, s));
    HH_STEP(cudaMallocAsync(&d_tw, sizeof(float) * tw.size(), s));
    HH_STEP(cudaMallocAsync(&d_cnt, sizeof(int64_t) * hh::CNT_N, s));
    const void* echo = echo_c64;
    if (host_echo) {
        HH_STEP(cudaMallocAsync(&d_echo, 8 * (size_t)n_pos * n_f, s));
        HH_STEP(cudaMemcpyAsync(d_echo, echo_c64, 8 * (size_t)n_pos * n_f, cudaMemcpyHostToDevice, s));
        echo = d_echo;
    }
    HH_STEP(cudaMemcpyAsync(d_traj, traj_xyz, sizeof(double) * 3 * n_pos, cudaMemcpyHostToDevice, s));
    HH_STEP(cudaMemcpyAsync(d_tw, tw.data(), sizeof(float) * tw.size(), cudaMemcpyHostToDevice, s));
    HH_STEP(cudaMemsetAsync(d_cnt, 0, sizeof(int64_t) * hh::CNT_N, s));
    HH_STEP(cudaMemsetAsync(grad_traj, 0, sizeof(double) * 3 * (size_t)n_pos, s));
    HH_STEP(hh::launch_rc(echo, nullptr, n_pos, n_f, tmp.n_fft, tmp.gate0, tmp.gate_n, d_tw, d_prof, nullptr,
                          cuda_stream));
    HH_STEP(hh::launch_bpa_grad(static_cast<const double*>(d_traj), n_pos, d_prof, kc, *grid, grad_image_c64,
                                grad_traj, d_cnt, cuda_stream));
    release();
#undef HH_STEP
    return HH_OK;
}

int bpa_adjoint(const double* traj_xyz, int64_t n_pos, const double* freqs_hz, int32_t n_f, const hh_grid* grid,
                const hh_config* cfg, const void* image_c64, void* echo_c64, void* cuda_stream) {
    int st = hh::validate_inputs(traj_xyz, n_pos, freqs_hz, n_f, grid, cfg, false);
    if (st != HH_OK) return st;
    if (!image_c64 || !echo_c64) return HH_ERR_ARG;
    if (is_host_pointer(image_c64) || is_host_pointer(echo_c64)) return HH_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    hh_plan tmp;
    hh::direct_bpa_setup(traj_xyz, n_pos, freqs_hz, n_f, grid, cfg, tmp);
    const hh::KConst kc = hh::make_kconst(&tmp);
    std::vector<float> tw = hh::twiddle_table(tmp.n_fft);
    void *d_traj = nullptr, *d_bins = nullptr, *d_tw = nullptr, *d_cnt = nullptr;
    auto release = [&]() {
        for (void* b : {d_traj, d_bins, d_tw, d_cnt})
            if (b) cudaFreeAsync(b, s);
    };
#define HH_STEP(call)                          \
    do {                                       \
        cudaError_t e_ = (cudaError_t)(call);  \
        if (e_ != cudaSuccess) {               \
            release();                         \
            return fail_cuda(e_);              \
        }                                      \
    } while (0)
    const size_t bins_bytes = 8 * (size_t)n_pos * (size_t)(tmp.gate_n + 1);
    HH_STEP(cudaMallocAsync(&d_traj, sizeof(double) * 3 * n_pos, s));
    HH_STEP(cudaMallocAsync(&d_bins, bins_bytes, s));
    HH_STEP(cudaMallocAsync(&d_tw, sizeof(float) * tw.size(), s));
    HH_STEP(cudaMallocAsync(&d_cnt, sizeof(int64_t) * hh::CNT_N, s));
    HH_STEP(cudaMemcpyAsync(d_traj, traj_xyz, sizeof(double) * 3 * n_pos, cudaMemcpyHostToDevice, s));
    HH_STEP(cudaMemcpyAsync(d_tw, tw.data(), sizeof(float) * tw.size(), cudaMemcpyHostToDevice, s));
    HH_STEP(cudaMemsetAsync(d_cnt, 0, sizeof(int64_t) * hh::CNT_N, s));
    HH_STEP(cudaMemsetAsync(d_bins, 0, bins_bytes, s));
    HH_STEP(hh::launch_bpa_adjoint(static_cast<const double*>(d_traj), n_pos, n_f, kc, *grid, image_c64, d_bins, d_tw,
                                   tmp.n_fft, tmp.gate0, tmp.gate_n, echo_c64, d_cnt, cuda_stream));
    release();
#undef HH_STEP
    return HH_OK;
}

int hhffbp_plan_preimages(const hh_plan* p, int64_t node, const double* targets, int64_t n, double* out,
                          void* cuda_stream) {
    if (!p || !targets || !out || n < 0) return HH_ERR_ARG;
    if (!p->on_device) return HH_ERR_HOST_ONLY;
    if (node < 0 || node >= p->level_start[p->n_levels - 1]) return HH_ERR_ARG;  // non-root nodes only
    if (n == 0) return HH_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    void *d_t = nullptr, *d_o = nullptr;
    cudaError_t e = cudaMalloc(&d_t, sizeof(double) * 3 * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_o, sizeof(double) * 4 * n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_t, targets, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = (cudaError_t)hh::launch_preimage_probe(p, hh::make_kconst(p), (int)node, static_cast<const double*>(d_t), n,
                                                   static_cast<double*>(d_o), cuda_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_o, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_t);
    cudaFree(d_o);
    return e == cudaSuccess ? HH_OK : fail_cuda(e);
}

int hhffbp_plan_tile_fill(const hh_plan* p, int32_t level, int64_t* hist, void* cuda_stream) {
    if (!p || !hist) return HH_ERR_ARG;
    if (!p->on_device) return HH_ERR_HOST_ONLY;
    if (level < 0 || level >= p->n_levels - 1) return HH_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    void* d_h = nullptr;
    cudaError_t e = cudaMalloc(&d_h, sizeof(int64_t) * 257);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_h, 0, sizeof(int64_t) * 257, s);
    if (e == cudaSuccess) e = (cudaError_t)hh::launch_tile_fill(p, level, static_cast<unsigned long long*>(d_h), cuda_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hist, d_h, sizeof(int64_t) * 257, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_h);
    return e == cudaSuccess ? HH_OK : fail_cuda(e);
}

}  // extern "C"

namespace {
// The demand passes of hhffbp_form_image (need masks and preimages of every non-root level,
// the leaves' included) for the adjoint traversal, after clearing the counters.
int adjoint_prologue(hh_plan* p, const hh::KConst& kc, cudaStream_t s) {
    HH_CUDA(cudaMemsetAsync(p->d_counters, 0, sizeof(int64_t) * hh::CNT_N, s));
    if (p->n_levels < 2) return HH_OK;
    void* st = reinterpret_cast<void*>(s);
    for (int l = 0; l + 1 < p->n_levels; ++l) HH_LAUNCH(hh::launch_tile_refs(p, kc, l, st));
    HH_CUDA(cudaMemsetAsync(p->d_need, 0, sizeof(uint32_t) * (size_t)p->need_total, s));
    HH_LAUNCH(hh::launch_need_final(p, kc, st));
    for (int l = p->n_levels - 2; l >= 1; --l) HH_LAUNCH(hh::launch_need_level(p, kc, l, st));
    HH_LAUNCH(hh::launch_need_leaf(p, kc, st));
    return HH_OK;
}
}  // namespace

extern "C" {

int hhffbp_adjoint(const hh_plan* cp, const void* image_c64, void* echo_c64, void* cuda_stream) {
    if (!cp || !image_c64 || !echo_c64) return HH_ERR_ARG;
    if (!cp->on_device) return HH_ERR_HOST_ONLY;
    hh_plan* p = const_cast<hh_plan*>(cp);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    const int64_t n_vox = (int64_t)p->grid.nx * p->grid.ny * p->grid.nz;
    const bool host_img = is_host_pointer(image_c64), host_echo = is_host_pointer(echo_c64);
    const void* image = image_c64;
    void* echo = echo_c64;
    if (host_img) {
        HH_CUDA(cudaMemcpyAsync(p->d_image_stage, image_c64, 8 * (size_t)n_vox, cudaMemcpyHostToDevice, s));
        image = p->d_image_stage;
    }
    if (host_echo) echo = p->d_echo_stage;
    const hh::KConst kc = hh::make_kconst(p);
    if (int r = adjoint_prologue(p, kc, s)) return r;
    // range-bin sums B_i in the profile buffer (unused by the adjoint otherwise)
    HH_CUDA(cudaMemsetAsync(p->d_prof, 0, 8 * (size_t)p->n_pos * (size_t)(p->gate_n + 1), s));
    HH_LAUNCH(hh::launch_adjoint_traversal(p, kc, image, p->d_prof, nullptr, cuda_stream));
    HH_LAUNCH(hh::launch_rc_adj(p->d_prof, static_cast<const int64_t*>(p->d_perm), p->n_pos, p->n_f, p->n_fft,
                                p->gate0, p->gate_n, p->d_twiddle, echo, cuda_stream));
    if (host_echo)
        HH_CUDA(cudaMemcpyAsync(echo_c64, echo, 8 * (size_t)p->n_pos * p->n_f, cudaMemcpyDeviceToHost, s));
    p->last_stream = cuda_stream;
    return HH_OK;
}

int hhffbp_traj_gradient(const hh_plan* cp, const void* echo_c64, const void* grad_image_c64, double* grad_traj,
                         void* cuda_stream) {
    if (!cp || !echo_c64 || !grad_image_c64 || !grad_traj) return HH_ERR_ARG;
    if (!cp->on_device) return HH_ERR_HOST_ONLY;
    if (is_host_pointer(grad_image_c64) || is_host_pointer(grad_traj)) return HH_ERR_ARG;
    hh_plan* p = const_cast<hh_plan*>(cp);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    const void* echo = echo_c64;
    if (is_host_pointer(echo_c64)) {
        HH_CUDA(cudaMemcpyAsync(p->d_echo_stage, echo_c64, 8 * (size_t)p->n_pos * p->n_f, cudaMemcpyHostToDevice, s));
        echo = p->d_echo_stage;
    }
    const hh::KConst kc = hh::make_kconst(p);
    if (int r = adjoint_prologue(p, kc, s)) return r;
    HH_CUDA(cudaMemsetAsync(grad_traj, 0, sizeof(double) * 3 * (size_t)p->n_pos, s));
    HH_LAUNCH(hh::launch_rc(echo, static_cast<const int64_t*>(p->d_perm), p->n_pos, p->n_f, p->n_fft, p->gate0,
                            p->gate_n, p->d_twiddle, p->d_prof, nullptr, cuda_stream));
    HH_LAUNCH(hh::launch_adjoint_traversal(p, kc, grad_image_c64, nullptr, grad_traj, cuda_stream));
    p->last_stream = cuda_stream;
    return HH_OK;
}

int hh_mip(const void* image_c64, int32_t nx, int32_t ny, int32_t nz, int32_t axis, float* out, void* cuda_stream) {
    if (!image_c64 || !out || nx <= 0 || ny <= 0 || nz <= 0 || axis < 0 || axis > 2) return HH_ERR_ARG;
    if (is_host_pointer(image_c64) || is_host_pointer(out)) return HH_ERR_ARG;
    HH_LAUNCH(hh::launch_mip(image_c64, nx, ny, nz, axis, out, cuda_stream));
    return HH_OK;
}

int hh_release_cached_memory(void) {
    BlockCache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto& kv : c.free_blocks) {
        cudaSetDevice(kv.first.first);
        cudaFree(kv.second);
        c.sizes.erase(kv.second);
    }
    c.free_blocks.clear();
    c.cached_bytes = 0;
    cudaSetDevice(cur);
    return HH_OK;
}

const char* hh_status_string(int status) {
    switch (status) {
        case HH_OK: return "ok";
        case HH_ERR_ARG: return "invalid argument";
        case HH_ERR_FREQ_NONUNIFORM: return "frequencies are not equidistant and increasing";
        case HH_ERR_OOM: return "out of memory";
        case HH_ERR_CUDA: return "CUDA error";
        case HH_ERR_PLAN_NONCONVERGED: return "preimage solver did not converge";
        case HH_ERR_DEVICE_FLAG: return "a kernel raised an error counter";
        case HH_ERR_UNIMPLEMENTED: return "not implemented";
        case HH_ERR_HOST_ONLY: return "plan has no device state (built host-only)";
        case HH_ERR_SCRATCH_LIMIT: return "problem exceeds the fixed workspace of bpa_form_image_noalloc";
        default: return "unknown status";
    }
}

int hh_last_cuda_error(void) { return g_last_cuda; }

long long hh_kernel_launches(void) { return hh::g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
