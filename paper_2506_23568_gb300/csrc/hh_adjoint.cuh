// Adjoint (reprojection: image -> echoes) and position gradient of the fast method, as
// kernels in the translation unit of hh_kernels.cu (they share its device helpers).
//
// The forward map of hhffbp_form_image is linear in the echo: range compression
// (Eq. eq2_rangecompression), leaf subimages (Eqs. eq2_bpatimedomain, eq_sdc_mul,
// eq_sdc_phi), merges and the final level (Sec. III, Sec. IV-A, Fig. 4), with an exact
// fallback wherever a footprint leaves a child's lattice or meets a sample the image does
// not need or cannot place.  Its conjugate transpose is taken step by step in reverse:
//   final:  x(p) -> each root child c: w e^{-j phi_c(p)} x(p) into the samples of c's
//           footprint, or (fallback) the BPA-RC adjoint of c's members at p;
//   merges: y = adj_P(q) at each needed, feasible parent sample q -> the same child step
//           with the phase difference Phi_c - Phi_P of the forward;
//   leaves: y = adj_L(q) -> the BPA-RC adjoint over the leaf's members at q: bins m0, m0+1
//           of member i get (1 - t, t) e^{-j (2 k_c dR_i - psi)} y;
//   range compression: s_i[n] = sum_m e^{-j theta_n m} B_i[m] (k_rc_adj).
// The interpolate/fall-back decision depends on geometry alone and is taken by the same
// device code as the forward's: the target pool of each level is set to 0 at needed,
// feasible samples and NaN elsewhere, so a footprint meets a NaN exactly where the
// forward's interpolation would.  Nothing of the forward's values is stored or recomputed:
// the position gradient with the plan held fixed (tree, lattices, preimages and subarray
// phases fixed; only the BPA-RC terms of leaves and fallbacks move with the positions)
// needs the same traversal and the range profiles of the echo alone.
//
// Accumulation uses atomics (shared-memory box sums, then one global atomic per box sample
// or window bin), so sums are not bit-reproducible between runs.

namespace {

// Where the BPA-RC terms of the traversal go.
struct AdjOut {
    float2* bins;          // adjoint: [n_pos][gate_n + 1] range-bin sums B_i (tree order)
    double* grad;          // gradient: [n_pos][3] dL/dp'_i (trajectory order)
    const int64_t* perm;   // tree slot -> trajectory index
    const float4* prof;    // gradient: the forward profiles (P[m], P[m+1] - P[m]) (tree order)
};

// One BPA-RC term of member i (tree slot) at point pc (node frame, |pc| = Rc, local SDC phase
// psi, stored-bin coordinate muc of Rc), v = node centre - p'_i (and |v|^2 / 2), with y the
// adjoint value of the node's subimage at pc.  GRAD false: B_i[m0], B_i[m0 + 1] += (1 - t, t)
// e^{-j th} y, th = 2 k_c dR - psi.  GRAD true: returns in g the gradient of
// Re[conj(y) e^{j th} lerp] with respect to p'_i, -Re[conj(y) e^{j th} (j 2 k_c lerp + dP / dR)]
// (pc + v) / R (pc + v = p - p'_i).
template <bool GRAD>
__device__ __forceinline__ void bpa_term_adj(const AdjOut& ao, const KConst& k, int64_t i, float4 v, float3 pc,
                                             float Rc2, float Rc, float psi, float muc, float2 y, float g[3],
                                             int& miss) {
    const float nh = fmaf(pc.x, v.x, fmaf(pc.y, v.y, fmaf(pc.z, v.z, v.w)));
    const float R2 = fmaf(2.f, nh, Rc2);
    const float yr = rsqrtf(R2);
    const float R = R2 * yr;
    const float d0 = R - Rc;
    const float dR = fmaf(fmaf(-d0, fmaf(0.5f, R, 0.5f * Rc), nh), yr, d0);
    float s, c;
    sincos_2pi_reduced(fmaf(k.two_kc, dR, -psi), &s, &c);
    const float mu = fmaf(dR, k.inv_dR, muc);
    if (!k.wrap && !(mu >= 0.f && mu < (float)(k.gate_n - 1))) {  // outside the stored gate: not expected
        ++miss;
        if (GRAD) g[0] = g[1] = g[2] = 0.f;
        return;
    }
    const float fl = floorf(mu);
    const float t = mu - fl;
    int m = (int)fl;
    if (k.wrap) m &= (k.gate_n - 1);
    if (!GRAD) {
        const float2 cv = make_float2(fmaf(y.x, c, y.y * s), fmaf(y.y, c, -y.x * s));  // e^{-j th} y
        float2* row = ao.bins + i * (int64_t)(k.gate_n + 1);
        atomicAdd(&row[m].x, (1.f - t) * cv.x);
        atomicAdd(&row[m].y, (1.f - t) * cv.y);
        atomicAdd(&row[m + 1].x, t * cv.x);
        atomicAdd(&row[m + 1].y, t * cv.y);
    } else {
        const float4 Q = __ldg(ao.prof + i * (int64_t)k.gate_n + m);
        const float Lx = fmaf(t, Q.z, Q.x), Ly = fmaf(t, Q.w, Q.y);
        const float Dx = fmaf(-k.two_kc, Ly, Q.z * k.inv_dR), Dy = fmaf(k.two_kc, Lx, Q.w * k.inv_dR);
        const float Ex = c * Dx - s * Dy, Ey = fmaf(c, Dy, s * Dx);
        const float coef = -fmaf(y.x, Ex, y.y * Ey) * yr;  // -Re(conj(y) E) / R
        g[0] = coef * (pc.x + v.x);
        g[1] = coef * (pc.y + v.y);
        g[2] = coef * (pc.z + v.z);
    }
}

// Adjoint of block_fallback: for every thread with `want`, the BPA-RC adjoint (or gradient)
// of child C's members at pc (C's frame) with value y.  The wanting threads' points are
// compacted into slots 0 .. total-1 (shared memory), and each thread takes whole members.
// Adjoint: the points in range order, each member's terms accumulated bin by bin and added to
// its range-bin sums once per run of a bin.  Gradient: each member's gradient summed over all
// points in registers, then one FP64 atomic per axis.  All threads of the block must call it;
// scratch holds 8 x 256 float2 and s_wc 8 ints.
template <bool GRAD>
__device__ void block_fallback_adj(const DNode& C, const KConst& k, bool want, float3 pc, float2 y,
                                   const float4* __restrict__ nodev, const AdjOut& ao, float2* scratch, int* s_wc,
                                   int& miss) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned mball = __ballot_sync(0xffffffffu, want);
    if (lane == 0) s_wc[warp] = __popc(mball);
    __syncthreads();
    int base = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
        const int cw = s_wc[w];
        base += w < warp ? cw : 0;
        total += cw;
    }
    if (total == 0) return;  // the same for every thread of the block
    float4* s_pt = reinterpret_cast<float4*>(scratch);  // point, |point|
    float2* s_ps = scratch + 2 * kThreads;              // psi, range-bin coordinate
    float2* s_y = scratch + 3 * kThreads;               // adjoint value
    const int slot = base + __popc(mball & ((1u << lane) - 1u));
    if (want) {
        const float Rc2 = fmaf(pc.x, pc.x, fmaf(pc.y, pc.y, pc.z * pc.z));
        const float Rc = Rc2 * rsqrtf(Rc2);
        s_pt[slot] = make_float4(pc.x, pc.y, pc.z, Rc);
        s_ps[slot] = make_float2(local_psi(node_f(C), k, pc, Rc), fmaf(Rc, k.inv_dR, -(float)k.gate0));
        s_y[slot] = y;
    }
    __syncthreads();
    if (GRAD) {
        // A member per thread: its gradient is summed in registers over the block's points (read
        // from shared memory by every lane alike), then added with one FP64 atomic per axis.
        for (int i = C.mem_begin + (int)threadIdx.x; i < C.mem_end; i += kThreads) {
            const float4 v = __ldg(nodev + i);
            float g3[3] = {0.f, 0.f, 0.f};
            for (int pt = 0; pt < total; ++pt) {
                const float4 q = s_pt[pt];
                const float2 ps = s_ps[pt], yv = s_y[pt];
                float gr[3];
                bpa_term_adj<true>(ao, k, i, v, make_float3(q.x, q.y, q.z), q.w * q.w, q.w, ps.x, ps.y, yv, gr, miss);
                g3[0] += gr[0];
                g3[1] += gr[1];
                g3[2] += gr[2];
            }
            double* gi = ao.grad + 3 * ao.perm[i];
            atomicAdd(gi, (double)g3[0]);
            atomicAdd(gi + 1, (double)g3[1]);
            atomicAdd(gi + 2, (double)g3[2]);
        }
        __syncthreads();  // the scratch is reused by the caller
        return;
    }
    // The adjoint: the points sorted by their range to the node centre (rank by comparison,
    // ties by slot), then a member per thread; its terms are accumulated in two running bins
    // (m and m + 1 of the current lerp pair) and added to the member's range-bin sums only when
    // the bin changes, which for points in range order happens about once per bin.
    float4* s_pt2 = reinterpret_cast<float4*>(scratch + 4 * kThreads);
    float2* s_ps2 = scratch + 6 * kThreads;
    float2* s_y2 = scratch + 7 * kThreads;
    if (want) {
        const float key = s_pt[slot].w;
        int r = 0;
        for (int o = 0; o < total; ++o) {
            const float ko = s_pt[o].w;
            r += (ko < key) || (ko == key && o < slot);
        }
        s_pt2[r] = s_pt[slot];
        s_ps2[r] = s_ps[slot];
        s_y2[r] = s_y[slot];
    }
    __syncthreads();
    for (int i = C.mem_begin + (int)threadIdx.x; i < C.mem_end; i += kThreads) {
        const float4 v = __ldg(nodev + i);
        float2* row = ao.bins + (int64_t)i * (k.gate_n + 1);
        int cur = -2;  // bin of a0 (a1 belongs to cur + 1); -2: none
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
        auto flush = [&](int m, float2 a) {
            if (m >= 0 && (a.x != 0.f || a.y != 0.f)) {
                atomicAdd(&row[m].x, a.x);
                atomicAdd(&row[m].y, a.y);
            }
        };
        for (int pt = 0; pt < total; ++pt) {
            const float4 q = s_pt2[pt];
            const float2 ps = s_ps2[pt], yv = s_y2[pt];
            const float nh = fmaf(q.x, v.x, fmaf(q.y, v.y, fmaf(q.z, v.z, v.w)));
            const float R2 = fmaf(2.f, nh, q.w * q.w);
            const float yr = rsqrtf(R2);
            const float R = R2 * yr;
            const float d0 = R - q.w;
            const float dR = fmaf(fmaf(-d0, fmaf(0.5f, R, 0.5f * q.w), nh), yr, d0);
            float s, c;
            sincos_2pi_reduced(fmaf(k.two_kc, dR, -ps.x), &s, &c);
            const float mu = fmaf(dR, k.inv_dR, ps.y);
            if (!k.wrap && !(mu >= 0.f && mu < (float)(k.gate_n - 1))) {  // outside the stored gate: not expected
                ++miss;
                continue;
            }
            const float fl = floorf(mu);
            const float t = mu - fl;
            int m = (int)fl;
            if (k.wrap) m &= (k.gate_n - 1);
            const float2 cv = make_float2(fmaf(yv.x, c, yv.y * s), fmaf(yv.y, c, -yv.x * s));  // e^{-j th} y
            if (m != cur) {
                if (m == cur + 1) {  // the pair moved up one bin: a0 is complete
                    flush(cur, a0);
                    a0 = a1;
                } else {
                    flush(cur, a0);
                    flush(cur + 1, a1);
                    a0 = make_float2(0.f, 0.f);
                }
                a1 = make_float2(0.f, 0.f);
                cur = m;
            }
            a0.x = fmaf(1.f - t, cv.x, a0.x);
            a0.y = fmaf(1.f - t, cv.y, a0.y);
            a1.x = fmaf(t, cv.x, a1.x);
            a1.y = fmaf(t, cv.y, a1.y);
        }
        flush(cur, a0);
        flush(cur + 1, a1);
    }
    __syncthreads();  // the scratch is reused by the caller
}

// w x (|w x| < 2^26) rounded to an integer in the FMA pipe: the multiple of 16 nearest to
// w x by the magic constant 1.5 * 2^27 (whose ulp is 16), then the exact residual (one FMA,
// |.| <= 8) by kRoundMagic.
__device__ __forceinline__ int fixed_term(float w, float x) {
    constexpr float kMagic27 = 201326592.0f;  // 1.5 * 2^27
    const float hb = fmaf(w, x, kMagic27);
    const float r = fmaf(w, x, -(hb - kMagic27));
    return (__float_as_int(hb) - __float_as_int(kMagic27)) * 16 + (__float_as_int(r + kRoundMagic) - (int)kRoundBits);
}

// Adjoint of interp_children: for every active thread, each child's term of the forward,
// e^{j ph_c} I_c (ph_c the phase in s_wph), transposed: child c's samples in the footprint
// receive w e^{-j ph_c} y.  The union boxes of the active threads' footprints are staged from
// the children's target pool (0 at needed, feasible samples, NaN elsewhere, plus what other
// blocks have added so far) with the forward's geometry, so that a footprint is complete
// exactly when the forward's is; complete footprints scatter into the zeroed box, and every
// non-zero box sample is then added to the pool with one global atomic.  Children whose
// footprint is incomplete are flagged in fb_mask (bit ci) for the adjoint of the exact
// fallback.  All threads must call it.
//
// The box accumulates in 32-bit fixed point with integer shared-memory atomics (order-free
// sums, no retry loop under contention).  With max(|Re y| + |Im y|) < 2^e over the block's
// threads and tap weights of magnitude at most 1 (the least-squares weights peak at 1, at
// integer delays), a term times S = 2^(26 - e) is below 2^26 and is rounded to an integer
// (fixed_term): a resolution of 2^-26 of the block's largest value, near the FP32 rounding of
// the terms.  A box sample receives at most one term per thread, and in practice the sums
// stay far below 2^31; every atomic checks its own addition for a signed wrap, and a pass in
// which one wrapped is zeroed and scattered again at S = 2^(22 - e), where 256 terms stay
// below 2^30.  A non-finite y makes every staged box sample NaN.
template <int TAPS, bool LATTICE>
__device__ void adj_children(const DNode* __restrict__ nodes, int child0, int nch, float2* __restrict__ tpool,
                             const WPoly& wp, float2* s_stage, int* s_box, StageGeo* s_geo, bool active,
                             const float* s_wph, float2 y, unsigned& fb_mask) {
    static_assert(kThreads <= 256, "fixed-point box sums assume at most 256 terms per sample");
    __shared__ int s_npass;
    __shared__ unsigned s_ymax;
    for (int i = threadIdx.x; i < 6 * kMaxChild; i += blockDim.x) s_box[i] = (i % 6) < 3 ? INT_MAX : INT_MIN;
    if (threadIdx.x == 0) s_ymax = 0u;
    fb_mask = 0u;
    __syncthreads();
    const int t = threadIdx.x;
    {  // block maximum of |Re y| + |Im y| (non-negative floats order as their bits)
        const unsigned m = __reduce_max_sync(0xffffffffu, active ? __float_as_uint(fabsf(y.x) + fabsf(y.y)) : 0u);
        if ((threadIdx.x & 31) == 0) atomicMax(&s_ymax, m);
    }
    for (int ci = 0; ci < nch; ++ci) {
        const float wq[3] = {s_wph[(4 * ci + 0) * kThreads + t], s_wph[(4 * ci + 1) * kThreads + t],
                             s_wph[(4 * ci + 2) * kThreads + t]};
        int base[3] = {0, 0, 0};
        const bool inside = active && footprint_base<TAPS>(nodes[child0 + ci], wq, base);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int lo = __reduce_min_sync(0xffffffffu, inside ? base[d] : INT_MAX);
            const int hi = __reduce_max_sync(0xffffffffu, inside ? base[d] + TAPS - 1 : INT_MIN);
            if ((threadIdx.x & 31) == 0 && lo <= hi) {
                atomicMin(s_box + 6 * ci + d, lo);
                atomicMax(s_box + 6 * ci + 3 + d, hi);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // the forward's packing (interp_children): pitches and passes
        int pass = 0, used = 0;
        for (int ci = 0; ci < nch; ++ci) {
            const int* b = s_box + 6 * ci;
            StageGeo g;
            bool any = true;
            for (int d = 0; d < 3; ++d) {
                g.lo[d] = b[d];
                g.n[d] = b[3 + d] - b[d] + 1;
                any = any && b[d] <= b[3 + d];
            }
            if (LATTICE) {
                int q2 = any ? g.n[2] : 5;
                while (((1 << (q2 & 15)) & 0x0c60) == 0) ++q2;
                g.p2 = q2;
                g.p1 = any ? g.n[1] * q2 : 3;
                g.p1 += (3 - g.p1) & 15;
            } else {
                g.p2 = any ? g.n[2] | 1 : 1;
                g.p1 = any ? g.n[1] * g.p2 : 2;
                g.p1 += (2 - g.p1) & 3;
            }
            g.staged = any && (int64_t)g.n[0] * g.p1 <= kStageCap;
            const int size = g.staged ? g.n[0] * g.p1 : 0;
            if (used + size > kStageCap) {
                ++pass;
                used = 0;
            }
            g.pass = pass;
            g.off = used;
            used += size;
            s_geo[ci] = g;
        }
        s_npass = pass + 1;
    }
    __syncthreads();
    const int npass = s_npass;
    int2* s_acc = reinterpret_cast<int2*>(s_stage);  // the boxes in fixed point
    const float ymax = __uint_as_float(s_ymax);
    const bool finite = ymax <= FLT_MAX;
    int ex = 0;
    frexpf(finite ? ymax : 1.f, &ex);  // ymax < 2^ex
    const int sh = max(-122, min(126, 26 - ex));  // the fine scale; sh - 4 the safe one
    for (int ps = 0; ps < npass; ++ps) {
        // 1. stage this pass's boxes from the target pool (their NaN marks decide completeness)
        for (int ci = 0; ci < nch; ++ci) {
            const StageGeo& g = s_geo[ci];
            if (g.pass != ps || !g.staged) continue;
            const DNode& C = nodes[child0 + ci];
            const float2* src = tpool + C.pool_off;
            float2* dst = s_stage + g.off;
            for (BoxWalk it(g.n[1], g.n[2]); it.q0 < g.n[0]; it.next())
                dst[it.q0 * g.p1 + it.q1 * g.p2 + it.q2] =
                    src[((int64_t)(g.lo[0] + it.q0) * C.N[1] + (g.lo[1] + it.q1)) * C.N[2] + (g.lo[2] + it.q2)];
        }
        __syncthreads();
        unsigned ok_mask = 0u;  // children of this pass with a complete footprint
        if (active) {
            for (int ci = 0; ci < nch; ++ci) {
                const StageGeo& g = s_geo[ci];
                if (g.pass != ps) continue;
                const float wc[3] = {s_wph[(4 * ci + 0) * kThreads + t], s_wph[(4 * ci + 1) * kThreads + t],
                                     s_wph[(4 * ci + 2) * kThreads + t]};
                const DNode& C = nodes[child0 + ci];
                int base[3];
                if (!footprint_base<TAPS>(C, wc, base)) {
                    fb_mask |= 1u << ci;
                    continue;
                }
                float nan_sum = 0.f;  // NaN when some footprint sample is not a needed, feasible one
                for (int i0 = 0; i0 < TAPS; ++i0)
                    for (int i1 = 0; i1 < TAPS; ++i1)
#pragma unroll
                        for (int i2 = 0; i2 < TAPS; ++i2) {
                            const float2 v =
                                g.staged ? s_stage[g.off + (base[0] - g.lo[0] + i0) * g.p1 +
                                                   (base[1] - g.lo[1] + i1) * g.p2 + (base[2] - g.lo[2] + i2)]
                                         : tpool[C.pool_off + ((int64_t)(base[0] + i0) * C.N[1] + base[1] + i1) * C.N[2] +
                                                 base[2] + i2];
                            nan_sum += v.x - v.x;
                        }
                if (nan_sum == nan_sum)
                    ok_mask |= 1u << ci;
                else
                    fb_mask |= 1u << ci;
            }
        }
        __syncthreads();
        // 2. zero the staged boxes, 3. scatter the complete footprints into them (once more at the
        // safe scale if a fine-scale sum wrapped; the unstaged children go to the pool directly,
        // in the first round only)
        int shp = sh;
        for (int round = 0; round < 2; ++round, shp = sh - 4) {
            for (int ci = 0; ci < nch; ++ci) {
                const StageGeo& g = s_geo[ci];
                if (g.pass != ps || !g.staged) continue;
                for (int i = threadIdx.x; i < g.n[0] * g.p1; i += blockDim.x) s_acc[g.off + i] = make_int2(0, 0);
            }
            __syncthreads();
            const float scale = __int_as_float((127 + shp) << 23);
            int wrap = 0;  // sign bit set when one of this thread's atomic additions wrapped
            for (int ci = 0; ci < nch; ++ci) {
                if (!((ok_mask >> ci) & 1u)) continue;
                const StageGeo& g = s_geo[ci];
                if (round > 0 && !g.staged) continue;
                const DNode& C = nodes[child0 + ci];
                const float wc[3] = {s_wph[(4 * ci + 0) * kThreads + t], s_wph[(4 * ci + 1) * kThreads + t],
                                     s_wph[(4 * ci + 2) * kThreads + t]};
                float wt[3][TAPS];
                int base[3];
                footprint<TAPS>(C, wp, wc, wt, base);
                float sn, cs;
                sincos_2pi_reduced(s_wph[(4 * ci + 3) * kThreads + t], &sn, &cs);
                const float2 v = make_float2(fmaf(y.x, cs, y.y * sn), fmaf(y.y, cs, -y.x * sn));  // e^{-j ph} y
                if (g.staged) {
                    const float2 vs = make_float2(v.x * scale, v.y * scale);
                    int2* box = s_acc + g.off + (base[0] - g.lo[0]) * g.p1 + (base[1] - g.lo[1]) * g.p2 + (base[2] - g.lo[2]);
                    for (int i0 = 0; i0 < TAPS; ++i0)
                        for (int i1 = 0; i1 < TAPS; ++i1) {
                            const float w01 = wt[0][i0] * wt[1][i1];
                            int2* row = box + i0 * g.p1 + i1 * g.p2;
#pragma unroll
                            for (int i2 = 0; i2 < TAPS; ++i2) {
                                const float w = w01 * wt[2][i2];
                                const int qx = fixed_term(w, vs.x), qy = fixed_term(w, vs.y);
                                const int ox = atomicAdd(&row[i2].x, qx), oy = atomicAdd(&row[i2].y, qy);
                                const int sx = (int)((unsigned)ox + (unsigned)qx), sy = (int)((unsigned)oy + (unsigned)qy);
                                wrap |= ((sx ^ ox) & (sx ^ qx)) | ((sy ^ oy) & (sy ^ qy));
                            }
                        }
                } else {
                    for (int i0 = 0; i0 < TAPS; ++i0)
                        for (int i1 = 0; i1 < TAPS; ++i1) {
                            const float w01 = wt[0][i0] * wt[1][i1];
                            float2* row = tpool + C.pool_off +
                                          ((int64_t)(base[0] + i0) * C.N[1] + base[1] + i1) * C.N[2] + base[2];
#pragma unroll
                            for (int i2 = 0; i2 < TAPS; ++i2) {
                                const float w = w01 * wt[2][i2];
                                atomicAdd(&row[i2].x, w * v.x);
                                atomicAdd(&row[i2].y, w * v.y);
                            }
                        }
                }
            }
            if (!__syncthreads_or(wrap < 0)) break;
        }
        // 4. add the boxes to the pool
        const float unscale = __int_as_float((127 - shp) << 23);
        for (int ci = 0; ci < nch; ++ci) {
            const StageGeo& g = s_geo[ci];
            if (g.pass != ps || !g.staged) continue;
            const DNode& C = nodes[child0 + ci];
            float2* dstp = tpool + C.pool_off;
            for (BoxWalk it(g.n[1], g.n[2]); it.q0 < g.n[0]; it.next()) {
                const int2 q = s_acc[g.off + it.q0 * g.p1 + it.q1 * g.p2 + it.q2];
                if (q.x != 0 || q.y != 0 || !finite) {
                    float2* d = dstp + ((int64_t)(g.lo[0] + it.q0) * C.N[1] + (g.lo[1] + it.q1)) * C.N[2] +
                                (g.lo[2] + it.q2);
                    const float nan = __int_as_float(0x7fc00000);
                    atomicAdd(&d->x, finite ? (float)q.x * unscale : nan);
                    atomicAdd(&d->y, finite ? (float)q.y * unscale : nan);
                }
            }
        }
        __syncthreads();  // the staging buffer is reused by the next pass or the caller
    }
}

// Target pool of one non-root level: 0 at every needed sample whose preimage is feasible,
// NaN at every other lattice sample (one launch tile per block).
__global__ void __launch_bounds__(kThreads) k_adj_init(const DNode* __restrict__ nodes, TileMap tm,
                                                      const uint32_t* __restrict__ need,
                                                      const float4* __restrict__ xyz, float2* __restrict__ pool) {
    const DTile tile = tile_of(tm, nodes);
    const DNode n = nodes[tile.node];
    int a, b, c;
    lattice_index(threadIdx.x, tile, a, b, c);
    if (!(a < n.N[0] && b < n.N[1] && c < n.N[2])) return;
    const int64_t li = n.pool_off + ((int64_t)a * n.N[1] + b) * n.N[2] + c;
    const bool ok = need_bit(need, blockIdx.x) && xyz[li].w > 0.5f;
    pool[li] = ok ? make_float2(0.f, 0.f) : make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
}

// Adjoint of k_final: the image values x at the voxels of D to the root's children.
template <int TAPS, bool GRAD>
__global__ void __launch_bounds__(kThreads, 4) k_final_adj(const DNode* __restrict__ nodes, TileMap tm, int child0,
                                                          int nch, const float2* __restrict__ x_img,
                                                          float2* __restrict__ tpool, WPoly wp,
                                                          const float4* __restrict__ nodev, KConst k, hh_grid g,
                                                          AdjOut ao, unsigned long long* cnt) {
    extern __shared__ float4 s_dyn[];
    float2* s_stage = reinterpret_cast<float2*>(s_dyn);  // kStageCap samples
    __shared__ NRef s_ref[kMaxChild];
    __shared__ float s_phase[kMaxChild];
    __shared__ int s_box[6 * kMaxChild];
    __shared__ StageGeo s_geo[kMaxChild];
    __shared__ int s_wc[kThreads / 32];
    __shared__ float s_wph[kMaxChild * 4 * kThreads];
    if (nch > kMaxChild) {
        if (threadIdx.x == 0) count(cnt, CNT_ERROR, 1);
        return;
    }
    const DTile tile = tile_of(tm, nodes);
    const int lx = threadIdx.x & 7, ly = (threadIdx.x >> 3) & 7, lz = threadIdx.x >> 6;
    const int x = tile.o0 + lx, yy = tile.o1 + ly, z = tile.o2 + lz;
    // the forward's reference point and per-voxel coordinates (k_final)
    const double cxv = 0.5 * (min(tile.o0 + kTile0 - 1, g.nx - 1) - tile.o0),
                 cyv = 0.5 * (min(tile.o1 + kTile1 - 1, g.ny - 1) - tile.o1),
                 czv = 0.5 * (min(tile.o2 + kTile2 - 1, g.nz - 1) - tile.o2);
    const double ptx = g.x0 + (tile.o0 + cxv) * g.dx, pty = g.y0 + (tile.o1 + cyv) * g.dy,
                 ptz = g.z0 + (tile.o2 + czv) * g.dz;
    if ((int)threadIdx.x < 4 * nch) {  // the forward's references (k_final)
        const int ci = threadIdx.x >> 2;
        make_ref_quad(nodes[child0 + ci], k, ptx, pty, ptz, quad_mask(nch), s_ref[ci]);
        if ((threadIdx.x & 3) == 0) s_phase[ci] = (float)mod_2pi(s_ref[ci].phi);
    }
    __syncthreads();
    const float3 dl = make_float3((float)((lx - cxv) * g.dx), (float)((ly - cyv) * g.dy), (float)((lz - czv) * g.dz));
    const bool valid = x < g.nx && yy < g.ny && z < g.nz;
    float2 y = make_float2(0.f, 0.f);
    if (valid) y = x_img[((int64_t)z * g.ny + yy) * g.nx + x];
    const bool active = valid && (y.x != 0.f || y.y != 0.f);
    for (int ci = 0; ci < nch; ++ci) {
        float w[3] = {0.f, 0.f, 0.f}, ph = 0.f;
        if (valid) ph = s_phase[ci] + node_eval_ref(node_f(nodes[child0 + ci]), k, s_ref[ci], dl, w, true);
        s_wph[(4 * ci + 0) * kThreads + threadIdx.x] = w[0];
        s_wph[(4 * ci + 1) * kThreads + threadIdx.x] = w[1];
        s_wph[(4 * ci + 2) * kThreads + threadIdx.x] = w[2];
        s_wph[(4 * ci + 3) * kThreads + threadIdx.x] = ph;
    }
    unsigned fb_mask = 0u;
    adj_children<TAPS, false>(nodes, child0, nch, tpool, wp, s_stage, s_box, s_geo, active, s_wph, y, fb_mask);
    int miss = 0;
    for (int ci = 0; ci < nch; ++ci) {
        const bool want = active && ((fb_mask >> ci) & 1u);
        if (!__syncthreads_or(want)) continue;
        float s = 0.f, cc = 0.f;
        if (want) sincos_2pi_reduced(s_wph[(4 * ci + 3) * kThreads + threadIdx.x], &s, &cc);
        const NRef& R = s_ref[ci];
        const float2 yc = make_float2(fmaf(y.x, cc, y.y * s), fmaf(y.y, cc, -y.x * s));  // e^{-j ph} y
        block_fallback_adj<GRAD>(nodes[child0 + ci], k, want,
                                 make_float3(R.pc[0] + dl.x, R.pc[1] + dl.y, R.pc[2] + dl.z), yc, nodev, ao, s_stage,
                                 s_wc, miss);
    }
    count(cnt, CNT_GATE_MISS, (unsigned long long)miss);
}

// Adjoint of k_merge at level `level`: the adjoint values of its needed, feasible samples
// (spool) to its children's target pool (tpool).
template <int TAPS, bool GRAD>
__global__ void __launch_bounds__(kThreads, 4) k_merge_adj(const DNode* __restrict__ nodes, TileMap tm,
                                                          const float2* __restrict__ spool,
                                                          float2* __restrict__ tpool, WPoly wp,
                                                          const float4* __restrict__ nodev, KConst k,
                                                          const uint32_t* __restrict__ need,
                                                          const float4* __restrict__ xyz, AdjOut ao,
                                                          unsigned long long* cnt) {
    extern __shared__ float4 s_dyn[];
    float2* s_stage = reinterpret_cast<float2*>(s_dyn);  // kStageCap samples
    __shared__ NRef s_ref[1 + kMaxChild];
    __shared__ float s_phase[kMaxChild];
    __shared__ int s_first;
    __shared__ int s_box[6 * kMaxChild];
    __shared__ StageGeo s_geo[kMaxChild];
    __shared__ int s_wc[kThreads / 32], s_idx[kThreads];
    __shared__ float3 s_pt;
    __shared__ float s_wph[kMaxChild * 4 * kThreads];
    const DTile tile = tile_of(tm, nodes);
    const DNode P = nodes[tile.node];
    const NodeF pf = node_f(P);
    int a, b, c;
    lattice_index(threadIdx.x, tile, a, b, c);
    const bool valid0 = a < P.N[0] && b < P.N[1] && c < P.N[2];
    const bool needed0 = valid0 && need_bit(need, blockIdx.x);
    if (!__syncthreads_or(needed0)) return;
    int n_needed;
    const int slot = compact_tile(needed0, s_wc, s_idx, &n_needed);  // the forward's thread order
    const bool needed = slot >= 0;
    lattice_index(needed ? slot : 0, tile, a, b, c);
    const int64_t li = ((int64_t)a * P.N[1] + b) * P.N[2] + c;
    float3 p = make_float3(0.f, 0.f, 1.f);
    bool ok = false;
    if (needed) {
        const float4 q = xyz[P.pool_off + li];
        ok = q.w > 0.5f;
        p = make_float3(q.x, q.y, q.z);
    }
    // the forward's tile reference: the first feasible sample in thread order
    if (threadIdx.x == 0) s_first = kThreads;
    __syncthreads();
    if (ok) atomicMin(&s_first, (int)threadIdx.x);
    __syncthreads();
    if ((int)threadIdx.x == s_first) s_pt = p;
    __syncthreads();
    const bool any = s_first < kThreads;
    const int nch = P.nchild;
    if (nch > kMaxChild) {
        if (threadIdx.x == 0) count(cnt, CNT_ERROR, 1);
        return;
    }
    if (!any) return;  // block-uniform
    if ((int)threadIdx.x < 4 * (nch + 1)) {  // the forward's references (k_merge)
        const float3 pt = s_pt;
        const double px = P.cx + (double)pt.x, py = P.cy + (double)pt.y, pz = P.cz + (double)pt.z;
        const int xi = threadIdx.x >> 2;
        const DNode& X = xi == 0 ? P : nodes[P.child0 + xi - 1];
        make_ref_quad(X, k, px, py, pz, quad_mask(nch + 1), s_ref[xi]);
    }
    __syncthreads();
    if (threadIdx.x >= 1 && (int)threadIdx.x <= nch)
        s_phase[threadIdx.x - 1] = (float)mod_2pi(s_ref[threadIdx.x].phi - s_ref[0].phi);
    __syncthreads();
    float2 y = make_float2(0.f, 0.f);
    if (ok) {
        y = spool[P.pool_off + li];
        if (!(y.x == y.x && y.y == y.y)) y = make_float2(0.f, 0.f);  // never expected: feasible samples are finite
    }
    const bool active = ok && (y.x != 0.f || y.y != 0.f);
    const float3 pt = s_pt;
    const float3 dl = make_float3(p.x - pt.x, p.y - pt.y, p.z - pt.z);
    float wdum[3];
    const float dphiP = ok ? node_eval_ref(pf, k, s_ref[0], dl, wdum, false) : 0.f;
    for (int ci = 0; ci < nch; ++ci) {
        float w[3] = {0.f, 0.f, 0.f}, ph = 0.f;
        if (ok) ph = s_phase[ci] + node_eval_ref(node_f(nodes[P.child0 + ci]), k, s_ref[1 + ci], dl, w, true) - dphiP;
        s_wph[(4 * ci + 0) * kThreads + threadIdx.x] = w[0];
        s_wph[(4 * ci + 1) * kThreads + threadIdx.x] = w[1];
        s_wph[(4 * ci + 2) * kThreads + threadIdx.x] = w[2];
        s_wph[(4 * ci + 3) * kThreads + threadIdx.x] = ph;
    }
    unsigned fb_mask = 0u;
    adj_children<TAPS, true>(nodes, P.child0, nch, tpool, wp, s_stage, s_box, s_geo, active, s_wph, y, fb_mask);
    int miss = 0;
    for (int ci = 0; ci < nch; ++ci) {
        const bool want = active && ((fb_mask >> ci) & 1u);
        if (!__syncthreads_or(want)) continue;
        float s = 0.f, cc = 0.f;
        if (want) sincos_2pi_reduced(s_wph[(4 * ci + 3) * kThreads + threadIdx.x], &s, &cc);
        const NRef& R = s_ref[1 + ci];
        const float2 yc = make_float2(fmaf(y.x, cc, y.y * s), fmaf(y.y, cc, -y.x * s));  // e^{-j ph} y
        block_fallback_adj<GRAD>(nodes[P.child0 + ci], k, want,
                                 make_float3(R.pc[0] + dl.x, R.pc[1] + dl.y, R.pc[2] + dl.z), yc, nodev, ao, s_stage,
                                 s_wc, miss);
    }
    count(cnt, CNT_GATE_MISS, (unsigned long long)miss);
}

// Adjoint of k_stage0: the leaf samples' adjoint values (spool) to the BPA-RC adjoint (or
// gradient) of the leaf's members, block-cooperatively as for the exact fallbacks.
template <bool GRAD>
__global__ void __launch_bounds__(kThreads) k_leaf_adj(const DNode* __restrict__ nodes, TileMap tm,
                                                      const float2* __restrict__ spool,
                                                      const float4* __restrict__ leafv, KConst k,
                                                      const uint32_t* __restrict__ need,
                                                      const float4* __restrict__ xyz, AdjOut ao,
                                                      unsigned long long* cnt) {
    __shared__ float2 s_scr[8 * kThreads];
    __shared__ int s_wc[kThreads / 32];
    const DTile tile = tile_of(tm, nodes);
    const DNode n = nodes[tile.node];
    int a, b, c;
    lattice_index(threadIdx.x, tile, a, b, c);
    const bool valid = a < n.N[0] && b < n.N[1] && c < n.N[2];
    bool active = false;
    float3 p = make_float3(0.f, 0.f, 1.f);
    float2 y = make_float2(0.f, 0.f);
    if (valid && need_bit(need, blockIdx.x)) {
        const int64_t li = n.pool_off + ((int64_t)a * n.N[1] + b) * n.N[2] + c;
        const float4 q = xyz[li];
        if (q.w > 0.5f) {
            y = spool[li];
            p = make_float3(q.x, q.y, q.z);
            active = (y.x != 0.f || y.y != 0.f) && y.x == y.x && y.y == y.y;
        }
    }
    int miss = 0;
    block_fallback_adj<GRAD>(n, k, active, p, y, leafv, ao, s_scr, s_wc, miss);
    count(cnt, CNT_GATE_MISS, (unsigned long long)miss);
}

}  // namespace

// Preimages (and feasibility) of the needed leaf samples into the level-0 part of d_xyz:
// the demand pass's preimage step on the leaves, whose children it has none to mark.
int launch_need_leaf(const hh_plan* p, const KConst& kc, void* stream) {
    const int64_t ntiles = p->level_tiles[0];
    if (ntiles == 0 || p->n_levels < 2) return 0;
    float4* xyz = static_cast<float4*>(p->d_xyz) + p->xyz_base[0];
    k_need_level<6><<<(unsigned)ntiles, kThreads, 0, as_stream(stream)>>>(
        static_cast<const DNode*>(p->d_nodes), tile_map(p, 0), static_cast<const float*>(p->d_tile_ref), kc,
        zh_mid_of(p), need_of(p, 0), TileMap{}, nullptr, 0, xyz, static_cast<unsigned long long*>(p->d_counters));
    note_launch();
    return (int)cudaGetLastError();
}

// The adjoint traversal of hhffbp_form_image from the image d_img (complex64 [nz][ny][nx],
// device) down to the BPA-RC terms: into the range-bin sums d_bins ([n_pos][gate_n + 1],
// zeroed by the caller) when d_bins is set, else into the position gradient d_grad
// ([n_pos][3], trajectory order, zeroed by the caller; d_prof must hold the echo's
// profiles).  The demand passes (need masks, preimages of every non-root level) must have
// run on the stream.
int launch_adjoint_traversal(const hh_plan* p, const KConst& kc, const void* d_img, void* d_bins, double* d_grad,
                             void* stream) {
    const bool grad = d_bins == nullptr;
    AdjOut ao{static_cast<float2*>(d_bins), d_grad, static_cast<const int64_t*>(p->d_perm),
              static_cast<const float4*>(p->d_prof)};
    cudaStream_t s = as_stream(stream);
    const DNode* nodes = static_cast<const DNode*>(p->d_nodes);
    auto* cnt = static_cast<unsigned long long*>(p->d_counters);
    const int L = p->n_levels;
    if (L == 1) {  // no factorisation: the adjoint (gradient) of direct BPA over the positions in tree order
        if (!grad)
            return launch_bpa_adjoint_bins(static_cast<const double*>(p->d_mem_pos), p->n_pos, kc, p->grid, d_img,
                                           d_bins, p->d_counters, stream);
        return launch_bpa_grad_perm(static_cast<const double*>(p->d_mem_pos), p->n_pos, p->d_prof, kc, p->grid, d_img,
                                    d_grad, static_cast<const int64_t*>(p->d_perm), p->d_counters, stream);
    }
    if (int e = smem_optin()) return e;
    static int optin = 0;
    if (!optin) {
        const int smem = (int)(sizeof(float2) * kStageCap);
        cudaError_t e = cudaSuccess;
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_final_adj<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_final_adj<6, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_final_adj<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_final_adj<6, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_merge_adj<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_merge_adj<6, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_merge_adj<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_merge_adj<6, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return (int)e;
        optin = 1;
    }
    const size_t smem = sizeof(float2) * kStageCap;
    auto init = [&](int level) {
        const int64_t ntiles = p->level_tiles[level];
        if (ntiles == 0) return 0;
        k_adj_init<<<(unsigned)ntiles, kThreads, 0, s>>>(nodes, tile_map(p, level), need_of(p, level),
                                                         static_cast<const float4*>(p->d_xyz) + p->xyz_base[level],
                                                         static_cast<float2*>(p->d_pool[level & 1]));
        note_launch();
        return (int)cudaGetLastError();
    };
    // final level: the image to the root's children (level L - 2)
    if (int e = init(L - 2)) return e;
    {
        const auto& root = p->nodes[p->level_start[L - 1]];
        const int64_t ntiles = p->level_tiles[L - 1];
        float2* tpool = static_cast<float2*>(p->d_pool[(L - 2) & 1]);
        const float2* x = static_cast<const float2*>(d_img);
        const float4* nv = nodev_of(p, L - 2);
#define HH_FINAL_ADJ(T, G)                                                                                           \
    k_final_adj<T, G><<<(unsigned)ntiles, kThreads, smem, s>>>(nodes, tile_map(p, L - 1), (int)root.child0,         \
                                                              (int)root.nchild, x, tpool, p->wpoly, nv, kc, p->grid, \
                                                              ao, cnt)
        if (p->cfg.taps == 4) {
            if (grad) HH_FINAL_ADJ(4, true); else HH_FINAL_ADJ(4, false);
        } else {
            if (grad) HH_FINAL_ADJ(6, true); else HH_FINAL_ADJ(6, false);
        }
        note_launch();
#undef HH_FINAL_ADJ
        if (cudaError_t e = cudaGetLastError()) return (int)e;
    }
    // merges, top down: level l's adjoint values to level l - 1
    for (int l = L - 2; l >= 1; --l) {
        if (int e = init(l - 1)) return e;
        const int64_t ntiles = p->level_tiles[l];
        if (ntiles == 0) continue;
        const float2* spool = static_cast<const float2*>(p->d_pool[l & 1]);
        float2* tpool = static_cast<float2*>(p->d_pool[(l - 1) & 1]);
        const float4* xyz = static_cast<const float4*>(p->d_xyz) + p->xyz_base[l];
        const float4* nv = nodev_of(p, l - 1);
#define HH_MERGE_ADJ(T, G)                                                                                            \
    k_merge_adj<T, G><<<(unsigned)ntiles, kThreads, smem, s>>>(nodes, tile_map(p, l), spool, tpool, p->wpoly, nv, kc, \
                                                              need_of(p, l), xyz, ao, cnt)
        if (p->cfg.taps == 4) {
            if (grad) HH_MERGE_ADJ(4, true); else HH_MERGE_ADJ(4, false);
        } else {
            if (grad) HH_MERGE_ADJ(6, true); else HH_MERGE_ADJ(6, false);
        }
        note_launch();
#undef HH_MERGE_ADJ
        if (cudaError_t e = cudaGetLastError()) return (int)e;
    }
    // leaves: their adjoint values to the BPA-RC adjoint (gradient) of their members
    {
        const int64_t ntiles = p->level_tiles[0];
        if (ntiles > 0) {
            const float2* spool = static_cast<const float2*>(p->d_pool[0]);
            const float4* xyz = static_cast<const float4*>(p->d_xyz) + p->xyz_base[0];
            if (grad) {
                k_leaf_adj<true><<<(unsigned)ntiles, kThreads, 0, s>>>(nodes, tile_map(p, 0), spool, nodev_of(p, 0),
                                                                       kc, need_of(p, 0), xyz, ao, cnt);
                note_launch();
            } else {
                k_leaf_adj<false><<<(unsigned)ntiles, kThreads, 0, s>>>(nodes, tile_map(p, 0), spool, nodev_of(p, 0),
                                                                        kc, need_of(p, 0), xyz, ao, cnt);
                note_launch();
            }
            if (cudaError_t e = cudaGetLastError()) return (int)e;
        }
    }
    return 0;
}
