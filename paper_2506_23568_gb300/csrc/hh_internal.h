// Internal declarations shared by the host planner (hh_plan.cpp), the C ABI
// (hh_api.cpp) and the kernels (hh_kernels.cu).  Plain-old-data only in the
// structs that travel to the device.
#pragma once

#include <cstdint>
#include <functional>
#include <vector>

#include "../../include/hhffbp.h"

namespace hh {

constexpr double kC = 299792458.0;  // m/s
constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxLevels = 32;

// Device copy of a materialised node (every node of every level, root last).
// Lattice sample (iu, iv, in) of a node sits at (u, v, n) = lo + (iu, iv, in) / eta
// and is stored at pool[pool_off + (iu * N[1] + iv) * N[2] + in].
struct DNode {
    double cx, cy, cz;     // subarray centre ((a+b)/2, (e+g)/2) at the design height zbar
    double hxd, hyd;       // half extents (b-a)/2, (g-e)/2 in FP64 (tile references)
    float hx, hy;          // the same in FP32 (per-sample arithmetic)
    float C2;              // 4 (b-a)^2 + 4 (g-e)^2
    float usat, vsat;      // kmax/pi * (b-a), kmax/pi * (g-e): reach of u and v
    float lo[3];           // lattice origin in (u, v, n)
    float eta[3];          // lattice density per axis
    int32_t N[3];          // lattice size per axis
    int32_t mem_begin;     // tree-slot range of the members
    int32_t mem_end;
    int32_t child0;        // first child (node index), -1 for leaves
    int32_t nchild;
    int32_t pad_;
    int64_t pool_off;      // first sample in the node's level pool
};

// Interpolation weights as polynomials of x = 2 tau - 1 (tau the fractional
// index, in [0, 1)), degree 8, in even and odd parts per tap pair: with
// o_q = q - (taps/2 - 1) the tap offsets, w_q(x) = E_q(x^2) + x O_q(x^2) and
// w_{taps-1-q}(x) = E_q(x^2) - x O_q(x^2) for q < taps/2 (the least-squares
// weights satisfy w_{taps-1-q}(tau) = w_q(1 - tau)).  Coefficients lowest first.
constexpr int kPolyPairs = 3;  // taps / 2 for taps <= 6
struct WPoly {
    float e[kPolyPairs][5];
    float o[kPolyPairs][4];
};

// Launch tiles: 8 x 8 x 4 lattice samples (u, v, n) of one node, or 8 x 8 x 4 voxels (x, y, z).
constexpr int kTile0 = 8, kTile1 = 8, kTile2 = 4;
// Need masks: bit ((b mod 8) * 4 + c mod 4) of word (a mod 8) of a launch tile's
// eight 32-bit words marks lattice sample (a, b, c) as needed.
constexpr int kNeedWords = 8;
// A launch tile: a box of lattice samples of one node, or a box of voxels.
struct DTile {
    int32_t node;
    int32_t o0, o1, o2;    // first index per axis
};

// Where a launch finds its tiles (see tile_of in the kernels).
struct TileMap {
    const int64_t* off;    // per-node first tile (n_nodes + 1 entries), or nullptr for the voxel level
    const DTile* tiles;    // lattice levels: node and origin of every launch tile of the level
    int32_t node0, n_nodes;
    int32_t ntx, nty;      // voxel level: tiles along x and y
};

// Deferred exact fallbacks of one merge level: groups of points of one child
// (segments) whose member sums stage 0's kernel evaluates, and per output the
// records to add (fixes), in child order.
struct FbSeg {
    int32_t node, count;  // child node, points
    int64_t rec0;         // first record
};
struct FbRec {
    float x, y, z;  // point in the child's frame
    float c, s;     // exp(j theta): the remodulation of the child's term
    float pad;
};
struct FbFix {
    int64_t out;     // output sample (level pool or image voxel)
    int32_t rec[4];  // the deferred record of child 0..3, -1 when none
};
struct FbQueue {
    FbSeg* segs;
    FbRec* recs;
    void* vals;                   // float2 per record: exp(j theta) g_child(point)
    FbFix* fixes;
    unsigned long long* counts;   // [0] segments, [1] records, [2] fixes
    int64_t rec_cap;
};
constexpr int kDeferMin = 32;     // smaller groups are evaluated where they arise

// Host-side node record (the plan's own, FP64).
struct HNode {
    int level = 0, depth = 0, t = 0;
    int64_t begin = 0, end = 0;
    double rect[4] = {0, 0, 0, 0};  // x'min, x'max, y'min, y'max (after the minimum-extent rule)
    double zbar = 0, zmin = 0, zmax = 0;
    double lo[3] = {0, 0, 0}, eta[3] = {1, 1, 1};
    int64_t N[3] = {0, 0, 0};
    int64_t child0 = -1, nchild = 0;
    int64_t pool_off = 0;
};

// Scalar constants handed to every kernel by value.
struct KConst {
    float kmin, kmax, kc;
    float kmax_pi;         // kmax / pi
    float kc_half;         // kc / 2
    float kmax_quarter;    // kmax / 4
    float kdiff_4pi;       // (kmax - kmin) / (4 pi)
    float kmax_4pi;        // kmax / (4 pi)
    float kmin_4pi;        // kmin / (4 pi)
    float two_kc;          // 2 kc
    float inv_dR;          // 1 / dR
    float zh_floor;        // smallest height above a subarray's design plane for a lattice point
    int32_t gate0;         // first stored range bin
    int32_t gate_n;        // stored bins per position
    int32_t wrap;          // 1 when the gate is the whole period (index modulo gate_n)
    int32_t taps;
    int32_t fp32_refs;     // HH_FLAG_FP32_REFS: tile and node references in FP32 (precision study)
    double kc_d, kmax_d, kmin_d;  // FP64 copies for tile references
    double inv_dR_d;
};

// Device counters (int64): see hhffbp_plan_counters.
// CNT_NEEDED + level: samples evaluated at that level (the root: voxels).
enum Counter { CNT_FALLBACK = 0, CNT_INFEASIBLE = 1, CNT_NEWTON_FAIL = 2, CNT_GATE_MISS = 3, CNT_ERROR = 4,
               CNT_FALLBACK_UPDATES = 5, CNT_FB_DEFERRED = 6, CNT_FB_OVERFLOW = 7, CNT_NEEDED = 8,
               CNT_N = 8 + 2 * kMaxLevels };

}  // namespace hh

struct hh_plan {
    // inputs
    int64_t n_pos = 0;
    int32_t n_f = 0;
    hh_grid grid{};
    hh_config cfg{};
    std::vector<double> traj, freqs;
    // derived constants
    double kmin = 0, kmax = 0, kc = 0, dk = 0, dR = 0, zbar_all = 0, zh_floor = 0;
    int n_fft = 0;
    int64_t gate0 = 0, gate_n = 0;
    bool gate_wrap = false;
    int depth_leaves = 0, n_levels = 0;
    std::vector<int64_t> perm;
    std::vector<hh::HNode> nodes;
    std::vector<int64_t> level_start;        // n_levels + 1
    std::vector<int64_t> level_samples;      // per level (root: voxel count)
    std::vector<int64_t> level_tiles;        // launch tiles per level (root: voxel tiles)
    std::vector<int64_t> tile_off;           // per-node first tile, all non-root levels concatenated
    std::vector<int64_t> tile_off_base;      // per level: first entry in tile_off
    std::vector<int64_t> level_pairs;        // merge launches: tile pairs per level (see pair_off)
    std::vector<int64_t> pair_off;           // per-node first tile pair, all non-root levels concatenated
    std::vector<int64_t> pair_off_base;      // per level: first entry in pair_off
    hh::WPoly wpoly{};                       // interpolation weights (polynomials)
    int64_t max_pool = 0;
    // device state
    bool on_device = false;
    int device = 0;
    void* d_nodes = nullptr;
    void* d_tile_off = nullptr;  // int64 copy of tile_off
    void* d_mem_pos = nullptr;   // double[n_pos][3], tree order
    void* d_perm = nullptr;      // int64[n_pos]
    void* d_nodev = nullptr;     // float4[L-1][n_pos], tree order: node centre - p', |.|^2 / 2 (FP32)
    void* d_prof = nullptr;      // float4[n_pos][gate_n] (P[m], P[m+1] - P[m]), tree order
    void* d_prof2 = nullptr;     // float2[n_pos][(gate_n + 2) & ~1] P[m] alone (stage-0 windows)
    void* d_pool[2] = {nullptr, nullptr};
    void* d_twiddle = nullptr;   // float2[2 n_fft]
    void* d_counters = nullptr;  // int64[CNT_N]
    void* d_need = nullptr;      // uint32[8] bit mask per launch tile of every non-root level (need_base offsets)
    void* d_xyz = nullptr;       // float4 preimage (node frame, w = feasible) per sample of levels 1..L-2
    void* d_tile_ref = nullptr;      // float[16] warm start per launch tile of levels 0..L-2
    void* d_tiles = nullptr;         // DTile (node, origin) per launch tile of levels 0..L-2 (tile_ref_base)
    void* d_pair_off = nullptr;      // int64 copy of pair_off
    void* d_pairs = nullptr;         // int2 (tile, tile or -1) per tile pair of levels 0..L-2 (pair_base)
    std::vector<int64_t> pair_base;  // per level: first pair in d_pairs
    std::vector<int64_t> tile_ref_base;  // per level: first tile in d_tile_ref
    // deferred-fallback queue (one merge level at a time)
    void* d_fb_segs = nullptr;
    void* d_fb_recs = nullptr;
    void* d_fb_vals = nullptr;
    void* d_fb_fixes = nullptr;
    void* d_fb_counts = nullptr;
    int64_t fb_seg_cap = 0, fb_rec_cap = 0;
    std::vector<int64_t> need_base;  // per level: first word in d_need
    std::vector<int64_t> xyz_base;   // per level: first sample in d_xyz (levels >= 1)
    int64_t need_total = 0, xyz_total = 0;
    void* d_echo_stage = nullptr;   // complex64[n_pos][n_f] for host echoes
    void* d_image_stage = nullptr;  // complex64 image for host outputs
    int64_t workspace_bytes = 0;
    void* last_stream = nullptr;
    // stage profiling (hhffbp_plan_profile)
    bool profile = false;
    std::vector<void*> events;          // cudaEvent_t, created on demand
    std::vector<int> stage_kind, stage_level;
};

namespace hh {

// hh_plan.cpp
int validate_inputs(const double* traj, int64_t n_pos, const double* freqs, int32_t n_f, const hh_grid* grid,
                    const hh_config* cfg, bool need_plan);
int build_host_plan(hh_plan* p);
void range_constants(const double* freqs, int n_f, int range_os, double* kmin, double* kmax, double* kc,
                     double* dk, int* n_fft, double* dR);
std::vector<float> twiddle_table(int n_fft);
WPoly weight_poly(int taps, double eta);
// Runs f(i) for i in [0, n) on up to `threads` host threads (i = t, t + T, ...).
void parallel_for(int64_t n, int threads, const std::function<void(int64_t)>& f);

// hh_kernels.cu (launch wrappers; return cudaError_t as int)
int launch_rc(const void* echo, const int64_t* d_perm, int64_t n_pos, int n_f, int n_fft, int64_t gate0,
              int64_t gate_n, const void* d_twiddle, void* d_prof, void* d_prof2, void* stream);
int launch_bpa(const double* d_traj, int64_t n_pos, const void* d_prof, const KConst& kc, const hh_grid& g,
               void* d_image, void* d_counters, void* stream);
int launch_bpa_grad(const double* d_traj, int64_t n_pos, const void* d_prof, const KConst& kc, const hh_grid& g,
                    const void* d_gimg, double* d_grad, void* d_counters, void* stream);
int launch_bpa_adjoint(const double* d_traj, int64_t n_pos, int n_f, const KConst& kc, const hh_grid& g,
                       const void* d_img, void* d_bins, const void* d_twiddle, int n_fft, int64_t gate0, int64_t gate_n,
                       void* d_echo, void* d_counters, void* stream);
int launch_bpa_grad_perm(const double* d_traj, int64_t n_pos, const void* d_prof, const KConst& kc, const hh_grid& g,
                         const void* d_gimg, double* d_grad, const int64_t* d_perm, void* d_counters, void* stream);
int launch_bpa_adjoint_bins(const double* d_traj, int64_t n_pos, const KConst& kc, const hh_grid& g, const void* d_img,
                            void* d_bins, void* d_counters, void* stream);
int launch_rc_adj(const void* d_bins, const int64_t* d_perm, int64_t n_pos, int n_f, int n_fft, int64_t gate0,
                  int64_t gate_n, const void* d_twiddle, void* d_echo, void* stream);
int launch_need_leaf(const hh_plan* p, const KConst& kc, void* stream);
int launch_adjoint_traversal(const hh_plan* p, const KConst& kc, const void* d_img, void* d_bins, double* d_grad,
                             void* stream);
int launch_need_final(const hh_plan* p, const KConst& kc, void* stream);
int launch_need_level(const hh_plan* p, const KConst& kc, int level, void* stream);
int launch_tile_refs(const hh_plan* p, const KConst& kc, int level, void* stream);
int launch_tile_table(const hh_plan* p, void* stream);
int launch_stage0(const hh_plan* p, const KConst& kc, void* stream);
int launch_deferred(const hh_plan* p, const KConst& kc, int level, void* out, void* stream);
int launch_merge(const hh_plan* p, const KConst& kc, int level, void* stream);
int launch_final(const hh_plan* p, const KConst& kc, void* d_image, void* stream);
int launch_tile_fill(const hh_plan* p, int level, unsigned long long* d_hist, void* stream);
int launch_mip(const void* d_img, int nx, int ny, int nz, int axis, float* d_out, void* stream);
int launch_preimage_probe(const hh_plan* p, const KConst& kc, int node, const double* d_tgt, int64_t n, double* d_out,
                          void* stream);
KConst make_kconst(const hh_plan* p);

// hh_api.cpp: count one kernel launch of the library (hh_kernel_launches)
void note_launch();
// hh_api.cpp: record a CUDA error for hh_last_cuda_error() and map it to a status
int note_cuda_error(int cuda_error);
// hh_api.cpp: range constants and a range gate covering every (voxel, position) distance
// (the setup of the direct-BPA entry points)
void direct_bpa_setup(const double* traj_xyz, int64_t n_pos, const double* freqs_hz, int32_t n_f,
                      const hh_grid* grid, const hh_config* cfg, hh_plan& tmp);

}  // namespace hh
