// emt_step.cuh -- one transport step of every track in flight, as one
// kernel launch (arXiv:2203.09467 Sec. 2.1: one thread per track; Sec. 2.2:
// cross sections, continuous loss, discrete interactions, secondaries and
// cutoffs; Sec. 2.3: propagation; Sec. 2.4: scoring in kernels).
//
// Layout and scheduling (the paper's own design launches one kernel per
// model from the host; this one is GB300-first):
//  * Tracks live in two ping-pong structure-of-arrays buffers of Q slots.
//    Photons fill the front of a buffer, charged tracks the back, so one
//    step reads a dense, coalesced range per particle type and writes the
//    survivors and secondaries compactly into the other buffer: the step
//    is also the compaction and the particle-type partition.
//  * Work is handed out in chunks of blockDim.x tracks of one particle type
//    by an atomic dispenser, so every warp runs the photon or the charged
//    code path only, and blocks stay busy until the step is drained.
//  * Within a chunk the step runs in two phases.  Phase A (every lane, its
//    own track): cross sections, step limits, propagation, continuous loss,
//    boundary and process selection.  Tracks that interact are counting-
//    sorted by model into shared memory; phase B runs the samplers over the
//    sorted records, so a warp executes one model (or two, at a group
//    boundary) instead of every model its lanes happened to select.  This
//    is the paper's one-kernel-per-model idea (Sec. 2.2) done inside one
//    launch, without a round trip through device memory.
//  * Output slots are reserved once per warp: a shuffle prefix sum over the
//    lanes' photon and charged output counts and one atomicAdd per type.
//  * Capacity: a step whose outputs do not fit is discarded and the track
//    is copied unchanged (deferred, see k_step).  A deferred track keeps its
//    step counter, so its random stream and every result are unchanged (the
//    paper's out-of-memory robustness without loss of reproducibility,
//    Sec. 2.1).
#pragma once

#include "emt_device.cuh"

namespace emt {

template <typename R>
struct TrackReg {
    double x[3];
    R u[3];
    R T;
    uint64_t uid;
    uint32_t ev;
    uint32_t step;
    int type;
    int vol;
};

// outputs sharing one position, event and volume: survivor first, then
// secondaries
template <typename R>
struct StepOut {
    int n;
    int type[2];
    R T[2];
    R u[2][3];
    uint64_t uid[2];
    uint32_t step[2];
};

// Side effects of one step, staged in registers and applied only once the
// step is committed (a step whose outputs do not fit is discarded and the
// track is copied unchanged).  Every deposit of a step is made at the
// post-step point, in the volume the track was in before any boundary
// crossing: one histogram column per step.
struct Effects {
    double dep;   // deposited energy
    double esc;   // escaped energy
    double kill;  // energy of a track killed at the step limit
    int col;      // histogram column of the deposits
    bool finished;
    int live_delta;
    int substeps;  // RK4 evaluations of the step (field only)
};

// models, in the order of the cumulative selection per particle type
enum Model : int {
    kPhoto = 0,
    kCompton = 1,
    kPair = 2,
    kMoller = 3,
    kBhabha = 4,
    kBrems = 5,
    kAnnih = 6,
    kRayleigh = 7,
    kNumModels = 8,
    kNoInteraction = -1
};

template <typename R>
__device__ __forceinline__ void deposit_now(const Params<R>& p, uint32_t ev, int col, double e)
{
    if (!nonzero(e)) return;
    atomicAdd(&p.hist[(size_t)ev * p.hstride + col], e);
}

__device__ __forceinline__ double rest_energy(int type) { return type == 2 ? 2.0 * kMe : 0.0; }

// a track ended after `steps` steps: per-event counts, and the
// steps-per-track histogram by particle type when it is enabled
template <typename R>
__device__ __forceinline__ void finish_track(const Params<R>& p, uint32_t ev, int type, uint32_t steps)
{
    atomicAdd(&p.counts[2 * (size_t)ev + 0], (unsigned long long)steps);
    atomicAdd(&p.counts[2 * (size_t)ev + 1], 1ull);
    if (p.step_hist) {
        const uint32_t last = (uint32_t)(p.step_bins - 1);
        atomicAdd(&p.step_hist[(size_t)type * p.step_bins + (steps < last ? steps : last)], 1ull);
    }
}

// An event is finished when its live-track count reaches zero.  A thread
// adds its secondaries before removing its own track, so the count of an
// event cannot touch zero while one of its tracks is still alive.
template <typename R>
__device__ __forceinline__ void update_live(const Params<R>& p, uint32_t ev, int delta)
{
    if (delta == 0) return;
    int old = atomicAdd(&p.live[ev], delta);
    if (old + delta == 0) {
        unsigned k = atomicAdd(p.done_head, 1u);
        p.done_ring[k % (unsigned)p.max_events] = ev;
    }
}

template <typename R>
__device__ __forceinline__ void apply_effects(const Params<R>& p, uint32_t ev, int type, uint32_t steps,
                                              const Effects& fx)
{
    deposit_now(p, ev, fx.col, fx.dep);
    if (nonzero(fx.esc)) atomicAdd(&p.ledger[3 * (size_t)ev + 0], fx.esc);
    if (nonzero(fx.kill)) atomicAdd(&p.ledger[3 * (size_t)ev + 1], fx.kill);
    if (fx.finished) finish_track(p, ev, type, steps);
    update_live(p, ev, fx.live_delta);
}

// Phase A of one step of one track, in the order
//  1 cross sections at the pre-step energy   2 s_int = -ln(u0)/Sigma_tot
//  3 e+-: s_max = max(f R, min(R, r_final))  4 s_phys = min
//  5 propagate to min(s_phys, boundary), ties to the boundary
//  6 e+-: T' = R^-1(R(T) - s), deposit T - T'
//  7 e+- below the cut: deposit T' (+2 me for e+), track ends
//  8 boundary: logical volume update; leaving the world tallies escape
//  9 interaction: the model by u1 Sigma_tot against the cumulative pre-step
//    Sigma's; a model whose channel is closed at the post-loss energy makes
//    a null interaction.
// Returns the model to sample in phase B, or kNoInteraction.  `alive`
// reports whether the track survives phase A.
// G: geometry kind; X: the physics options (multiple scattering, angular
// distributions, Rayleigh) may be on (kernels without them carry no code
// for them)
template <int G, bool X, typename R>
__device__ __forceinline__ int transport_part(const Params<R>& p, TrackReg<R>& t, Effects& fx, bool& alive)
{
    fx.dep = 0.0;
    fx.esc = 0.0;
    fx.kill = 0.0;
    fx.finished = false;
    fx.live_delta = 0;
    fx.substeps = 0;
    const uint64_t event_id = p.event_id[t.ev];
    Draws dr;
    dr.init(p.seed, event_id, t.uid, t.step);
    const int mi = t.vol >= 0 ? p.lmat[t.vol] : -1;
    const bool matter = mi >= 0 && !p.vacuum[mi];
    const bool charged = t.type != 0;
    // photons: photo, Compton, pair (+ Rayleigh); e-: ioni, brems; e+: ioni,
    // brems, annihilation
    const int nproc = t.type == 1 ? 2 : ((X && t.type == 0 && (p.mask & kProcRayleigh)) ? 4 : 3);
    const size_t row = matter ? (size_t)(mi * 3 + t.type) * p.n_grid * kNq : 0;
    const R* tab = p.tab + row;
    const R* dtab = p.dtab + row;

    R sig[4] = {R(0), R(0), R(0), R(0)};
    R sig_tot = R(0);
    R Rng = R(0);
    Lookup<R> lk;
    lk.n = 0;
    lk.f = R(0);
    lk.clamp = -1;
    if (matter) {
        lk = locate_energy(p, t.T);
        sig[0] = xs_value(p, tab, dtab, lk, 0);
        sig[1] = xs_value(p, tab, dtab, lk, 1);
        sig_tot = sig[0] + sig[1];
        if (nproc >= 3) {
            sig[2] = xs_value(p, tab, dtab, lk, 2);
            sig_tot = sig_tot + sig[2];
        }
        if constexpr (X) {
            if (nproc == 4) {
                sig[3] = xs_value(p, tab, dtab, lk, 3);
                sig_tot = sig_tot + sig[3];
            }
        }
    }
    const R kInf = R(__longlong_as_double(0x7FF0000000000000ll));
    R s_int = kInf;
    int proc = nproc - 1;
    if (gt_zero(sig_tot)) {
        dr.next = 0;
        s_int = mdiv(-mlog(draw<R>(dr)), sig_tot);
        // 9, taken early: the model by draw 1 (the same Philox block as
        // draw 0) against the cumulative pre-step cross sections.  It reads
        // only pre-step values, so it is the choice the step makes if it
        // interacts (unused otherwise); taking it here frees the cross
        // sections and the draw state before the propagation.
        const R xsel = draw<R>(dr) * sig_tot;
        R c = R(0);
        for (int i = 0; i < nproc; ++i) {
            c += sig[i];
            if (lt_pos(xsel, c)) {
                proc = i;
                break;
            }
        }
    }
    R s_max = kInf;
    if (charged && matter) {
        Rng = range_value(p, tab, dtab, t.T, lk);
        R fr_lim = pfinal_range(p);
        R lim = lt_pos(Rng, fr_lim) ? Rng : fr_lim;
        R fr = pstep_frac(p) * Rng;
        s_max = lt_pos(lim, fr) ? fr : lim;
    }
    R s_phys = s_max;
    bool interact = false;
    if (lt_pos(s_int, s_max)) {
        s_phys = s_int;
        interact = true;
    }

    // 5: propagation (positions and boundary distances in FP64)
    double s;
    bool boundary = false;
    Exit e;
    const double s_physd = to_d(s_phys);
    if (!(charged && p.has_field)) {
        const double ud[3] = {to_d(t.u[0]), to_d(t.u[1]), to_d(t.u[2])};
        if constexpr (G == kGeomCylinders) {
            // cylinders (thick shells, navigation with square roots): a
            // physics step that ends more than the chord margin inside the
            // shell has an exit distance above s_phys by at least the
            // margin (far above its rounding): no boundary, exactly as the
            // full navigation would decide
            double x1[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) x1[a] = fma(s_physd, ud[a], t.x[a]);
            if (!chord_inside<G>(p, t.vol, t.x, x1)) {
                e = nav_exit<G>(p, t.vol, t.x, ud);
                boundary = le_pos(e.t, s_physd);
            }
            if (boundary) {
                s = e.t;
#pragma unroll
                for (int a = 0; a < 3; ++a) t.x[a] = fma(s, ud[a], t.x[a]);
                if (e.axis >= 0) t.x[e.axis] = e.plane;
            } else {
                s = s_physd;
#pragma unroll
                for (int a = 0; a < 3; ++a) t.x[a] = x1[a];
            }
        } else {
            // thin layers: most steps cross a plane; the navigation (with
            // its FP32 prefilter) is cheaper than a test that mostly fails
            e = nav_exit<G>(p, t.vol, t.x, ud);
            if (le_pos(e.t, s_physd)) {
                s = e.t;
                boundary = true;
            } else {
                s = s_physd;
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) t.x[a] = fma(s, ud[a], t.x[a]);
            if (boundary && e.axis >= 0) t.x[e.axis] = e.plane;
        }
    } else {
        double smax = s_physd;
        if (smax > p.max_field_step) {
            smax = p.max_field_step;
            interact = false;
        }
        // substeps of at most h_max = sqrt(8 r delta), r = p / (c |B|); at
        // most kMaxSubsteps of them
        const double Td = to_d(t.T);
        const double pm = msqrt(Td * (Td + 2.0 * kMe));
        const double hmax = msqrt(8.0 * mdiv(pm, kFieldC * p.bmag) * p.rk_delta);
        int nsub;
        double hs;
        if (smax > kMaxSubsteps * hmax) {
            nsub = kMaxSubsteps;
            hs = hmax;
            interact = false;
        } else {
            double ns = ceil(mdiv(smax, hmax));
            if (ns < 1.0) ns = 1.0;
            nsub = (int)ns;
            hs = mdiv(smax, ns);
        }
        bool crossed = false;
        s = propagate_field<G>(p, t.type == 1 ? -1 : 1, pm, t.vol, t.x, t.u, nsub, hs, &e, &crossed, &fx.substeps);
        boundary = crossed;
    }
    if (boundary) interact = false;
    fx.col = score_col(p, t.vol, t.x[2]);

    alive = true;
    const R T0 = t.T;
    // 6-7: continuous loss
    if (charged && matter) {
        R r = Rng - from_d<R>(s);
        R Tn = gt_zero(r) ? inv_range(p, tab, p.irs + (size_t)(mi * 3 + t.type) * p.n_grid, r, lk.n) : R(0);
        R ed = t.T - Tn;
        fx.dep = to_d(ed);  // 0 + ed: ed is never -0
        t.T = Tn;
        if (lt_pos(t.T, pcut(p, t.type))) {
            fx.dep += to_d(t.T) + rest_energy(t.type);
            alive = false;
        }
    }
    // 6b: multiple scattering at the post-step point (boundary steps too)
    if constexpr (X) {
        if (alive && charged && matter && (p.mask & kProcMsc) && gt_zero(s))
            msc_deflect(dr, T0, from_d<R>(s), from_d<R>(p.x0[mi]), t.u);
    }
    // 8: boundary
    if (alive && boundary) {
        t.vol = e.next;
        if (t.vol == kVolOut) {
            fx.esc = to_d(t.T) + rest_energy(t.type);
            alive = false;
        }
        return kNoInteraction;
    }
    if (!alive || !interact) return kNoInteraction;
    // 9: the model chosen above, and channels closed at the post-loss energy
    const R T = t.T;
    if (t.type == 0) {
        if (proc == 0) return T > from_d<R>(p.bk[mi]) ? kPhoto : kNoInteraction;
        if (proc == 1) return kCompton;
        if (X && proc == 3) return kRayleigh;
        return T > R(2.0 * kMe) ? kPair : kNoInteraction;
    }
    if (proc == 0) {
        if (t.type == 1) return T > R(2) * pcut(p, 1) ? kMoller : kNoInteraction;
        return T > pcut(p, 1) ? kBhabha : kNoInteraction;
    }
    if (proc == 1) return T > pcut(p, 0) ? kBrems : kNoInteraction;
    return kAnnih;
}

// step 10 for a track that did not interact: count the step, apply the
// step limit, and emit the survivor
template <typename R>
__device__ __forceinline__ void finish_step(const Params<R>& p, TrackReg<R>& t, bool alive, Effects& fx, StepOut<R>& o)
{
    t.step += 1;
    if (alive && (int)t.step >= p.max_steps) {
        fx.kill = to_d(t.T) + rest_energy(t.type);
        alive = false;
    }
    o.n = 0;
    if (alive) {
        o.type[0] = t.type;
        o.T[0] = t.T;
        o.u[0][0] = t.u[0];
        o.u[0][1] = t.u[1];
        o.u[0][2] = t.u[2];
        o.uid[0] = t.uid;
        o.step[0] = t.step;
        o.n = 1;
    } else {
        fx.finished = true;
        fx.live_delta = -1;
    }
}

// Phase B: sample model `m` for the post-loss state t (draws 2, 3, ... of
// the step), then step 10.  Secondaries below their cut deposit on the spot.
template <bool X, typename R>
__device__ __forceinline__ void interaction_part(const Params<R>& p, TrackReg<R>& t, int m, Effects& fx,
                                                 StepOut<R>& o)
{
    const bool angular = X && (p.mask & kProcAngular) != 0u;
    const uint64_t event_id = p.event_id[t.ev];
    Draws dr;
    dr.init(p.seed, event_id, t.uid, t.step);
    dr.next = 2;
    Products<R> pr;
    pr.n = 0;
    pr.local = R(0);
    pr.parent_alive = true;
    const R T = t.T;
    const R cut_e = pcut(p, 1), kc = pcut(p, 0);
    switch (m) {
    case kPhoto: sample_photo(dr, T, from_d<R>(p.bk[p.lmat[t.vol]]), t.u, pr, angular); break;
    case kCompton: sample_compton(dr, T, t.u, pr, t.T); break;
    case kPair: sample_pair(dr, T, t.u, pr, angular); break;
    case kMoller: sample_moller(dr, T, cut_e, t.u, pr, t.T); break;
    case kBhabha: sample_bhabha(dr, T, cut_e, t.u, pr, t.T); break;
    case kBrems: sample_brems(dr, T, kc, t.u, pr, t.T, angular); break;
    case kRayleigh:
        if constexpr (X) sample_rayleigh(dr, T, from_d<R>(p.ray_a[p.lmat[t.vol]]), t.u);
        break;
    default: sample_annih(dr, T, t.u, pr); break;
    }
    if (pr.local != R(0)) fx.dep += to_d(pr.local);
    // secondaries below their cut deposit on the spot (in the order k = 0, 1)
    bool keep[2] = {false, false};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (k < pr.n) {
            const int st = pr.type[k];
            if (lt_pos(pr.T[k], pcut(p, st)))
                fx.dep += to_d(pr.T[k]) + rest_energy(st);
            else
                keep[k] = true;
        }
    }
    bool alive = true;
    if (!pr.parent_alive) {
        alive = false;
    } else if (lt_pos(t.T, pcut(p, t.type))) {
        fx.dep += to_d(t.T) + rest_energy(t.type);
        alive = false;
    }
    const uint32_t parent_step = t.step;
    finish_step(p, t, alive, fx, o);
    // outputs: the survivor (slot 0), then the kept secondaries in order.
    // A surviving parent has at most one secondary, so every slot index
    // below is a constant (the outputs stay in registers).
    auto put = [&](int j, int k) {
        o.type[j] = pr.type[k];
        o.T[j] = pr.T[k];
        o.u[j][0] = pr.dir[k][0];
        o.u[j][1] = pr.dir[k][1];
        o.u[j][2] = pr.dir[k][2];
        o.uid[j] = child_uid(p.seed, event_id, t.uid, parent_step, (uint32_t)k);
        o.step[j] = 0;
    };
    if (o.n == 1) {
        if (keep[0]) {
            put(1, 0);
            o.n = 2;
        }
    } else if (keep[0]) {
        put(0, 0);
        o.n = 1;
        if (keep[1]) {
            put(1, 1);
            o.n = 2;
        }
    } else if (keep[1]) {
        put(0, 1);
        o.n = 1;
    }
    fx.live_delta += (int)keep[0] + (int)keep[1];
}

// Scheduling key of a charged track's next step in a field: an estimate,
// in FP32, of its number of RK4 substeps, ceil(s / h_max) with s the
// smallest of the free path (draw 0 of the step), the range limit, the
// field-step limits and, in a layer, the straight-line distance to the
// z plane ahead (curvature ignored), clamped to [1, kMaxSubsteps].  It only
// decides which lanes run together; the step itself recomputes everything
// in the method's own arithmetic.
template <typename R>
__device__ __forceinline__ int field_substeps_estimate(const Params<R>& p, const TrackReg<R>& t)
{
    const float T = est_f(t.T);
    const float pm = sqrtf(T * (T + 2.0f * (float)kMe));
    const float hmax = sqrtf(8.0f * (pm / ((float)kFieldC * (float)p.bmag)) * (float)p.rk_delta);
    float s = fminf((float)p.max_field_step, (float)kMaxSubsteps * hmax);
    const int mi = t.vol >= 0 ? p.lmat[t.vol] : -1;
    if (mi >= 0 && !p.vacuum[mi]) {
        const size_t row = (size_t)(mi * 3 + t.type) * p.n_grid * kNq;
        const R* tab = p.tab + row;
        const R* dtab = p.dtab + row;
        const Lookup<R> lk = locate_energy(p, t.T);
        const float rng = est_f(range_value(p, tab, dtab, t.T, lk));
        const float lim = fminf(rng, est_f(pfinal_range(p)));
        s = fminf(s, fmaxf(est_f(pstep_frac(p)) * rng, lim));
        float sig = est_f(xs_value(p, tab, dtab, lk, 0)) + est_f(xs_value(p, tab, dtab, lk, 1));
        if (t.type == 2) sig += est_f(xs_value(p, tab, dtab, lk, 2));
        if (sig > 0.0f) {
            Draws dr;
            dr.init(p.seed, p.event_id[t.ev], t.uid, t.step);
            dr.fill(0);
            const float u = __uint_as_float(0x3F800000u | (dr.w[1] >> 9)) - (1.0f - 0x1p-24f);
            s = fminf(s, -__logf(u) / sig);
        }
    }
    if (p.geom == kGeomLayers && t.vol >= 0) {
        // the straight-line distance to the layer's z plane ahead: the step
        // ends there after about that many substeps and one repeated one
        const float uz = est_f(t.u[2]);
        const float z = (float)t.x[2];
        float dz = 3.0e38f;
        if (uz > 0.0f) dz = ((float)p.zb[t.vol + 1] - z) / uz;
        if (uz < 0.0f) dz = (z - (float)p.zb[t.vol]) / -uz;
        s = fminf(s, fmaxf(dz, 0.0f) + hmax);
    }
    const float n = ceilf(s / hmax);
    return n < 1.0f ? 1 : (n > (float)kMaxSubsteps ? kMaxSubsteps : (int)n);
}

// RK4 evaluations of a warp's steps into the run's counter (field only;
// every lane of the warp calls it)
template <typename R>
__device__ __forceinline__ void count_substeps(const Params<R>& p, int lane, int substeps)
{
    if (!p.has_field) return;
    const unsigned v = __reduce_add_sync(0xFFFFFFFFu, (unsigned)substeps);
    if (lane == 0 && v) atomicAdd(&p.total_steps[3], (unsigned long long)v);
}

template <typename R>
__device__ __forceinline__ void load_track(const Tracks<R>& q, long long i, TrackReg<R>& t)
{
    t.x[0] = q.x[i];
    t.x[1] = q.y[i];
    t.x[2] = q.z[i];
    t.u[0] = q.ux[i];
    t.u[1] = q.uy[i];
    t.u[2] = q.uz[i];
    t.T = q.T[i];
    t.uid = q.uid[i];
    t.ev = q.ev[i];
    t.step = q.step[i];
    uint32_t tv = q.tv[i];
    t.type = tv_type(tv);
    t.vol = tv_vol(tv);
}

template <typename R>
__device__ __forceinline__ void store_track(const Tracks<R>& q, long long i, const double x[3], const R u[3], R T,
                                            uint64_t uid, uint32_t ev, uint32_t step, int type, int vol)
{
    q.x[i] = x[0];
    q.y[i] = x[1];
    q.z[i] = x[2];
    q.ux[i] = u[0];
    q.uy[i] = u[1];
    q.uz[i] = u[2];
    q.T[i] = T;
    q.uid[i] = uid;
    q.ev[i] = ev;
    q.step[i] = step;
    q.tv[i] = pack_tv(type, vol);
}

template <typename R>
__device__ __forceinline__ void copy_out(const TrackReg<R>& t, StepOut<R>& o)
{
    o.n = 1;
    o.type[0] = t.type;
    o.T[0] = t.T;
    o.u[0][0] = t.u[0];
    o.u[0][1] = t.u[1];
    o.u[0][2] = t.u[2];
    o.uid[0] = t.uid;
    o.step[0] = t.step;
}

// warp-aggregated reservation and store of each lane's outputs (all lanes
// of the warp call it); counts are packed as photons | charged << 16.
// With track selection on, eh (shared memory) counts the outputs' energy
// classes.  kMaxOut: the most outputs a lane can have (1 after the
// transport part, 2 after an interaction); the loops over the outputs are
// unrolled to it, so the outputs stay in registers.
template <int kMaxOut, typename R>
__device__ __forceinline__ void emit(const Params<R>& p, const Tracks<R>& qo, Counters* cout, int lane,
                                     const StepOut<R>& o, const double x[3], uint32_t ev, int vol,
                                     unsigned* eh = nullptr)
{
    int ng = 0, nc = 0;
#pragma unroll
    for (int k = 0; k < kMaxOut; ++k) {
        if (k < o.n) {
            if (o.type[k] == 0)
                ++ng;
            else
                ++nc;
        }
    }
    const int v = ng | (nc << 16);
    int incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off) incl += y;
    }
    const int excl = incl - v;
    const int tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (tot == 0) return;
    int baseG = 0, baseC = 0;
    if (lane == 31) {
        int tg = tot & 0xFFFF, tc = tot >> 16;
        if (tg) baseG = atomicAdd(&cout->n[0], tg);
        if (tc) baseC = atomicAdd(&cout->n[1], tc);
    }
    baseG = __shfl_sync(0xFFFFFFFFu, baseG, 31);
    baseC = __shfl_sync(0xFFFFFFFFu, baseC, 31);
    long long og = (long long)baseG + (excl & 0xFFFF);
    long long oc = (long long)baseC + (excl >> 16);
    const long long Q = p.Q;
#pragma unroll
    for (int k = 0; k < kMaxOut; ++k) {
        if (k >= o.n) break;
        long long dst;
        if (o.type[k] == 0) {
            dst = og++;
        } else {
            dst = Q - 1 - oc;
            ++oc;
        }
        if (dst < 0 || dst >= Q) {
            atomicOr(p.status, kStatusQueueOverflow);
            continue;
        }
        store_track(qo, dst, x, o.u[k], o.T[k], o.uid[k], ev, o.step[k], o.type[k], vol);
        if (eh) atomicAdd(&eh[energy_class(est_f(o.T[k]))], 1u);
    }
}

// Track selection (the paper's Sec. 3.2: preferring low-energy tracks keeps
// the number of tracks in flight, and so the capacity needed, down).  The
// lowest-energy class c* whose cumulative count over the input reaches
// max_active, and the quota of tracks of class c* that may still step.
// One warp computes it from the input slot's energy-class counts.
struct Selection {
    int cls;    // classes below step, above are held; kEBins: all step
    int quota;  // tickets of class cls that step
};

template <typename R>
__device__ __forceinline__ Selection select_threshold(const Params<R>& p, int cin, int lane, long long A)
{
    const unsigned* h = p.ehist + (size_t)cin * kEBins;
    unsigned c[kEBins / 32];
    long long local = 0;
#pragma unroll
    for (int k = 0; k < kEBins / 32; ++k) {
        c[k] = h[lane * (kEBins / 32) + k];
        local += c[k];
    }
    long long incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off) incl += y;
    }
    const unsigned reach = __ballot_sync(0xFFFFFFFFu, incl >= A);
    Selection sel;
    sel.cls = kEBins;
    sel.quota = 0;
    if (!reach) return sel;
    const int L = __ffs(reach) - 1;
    if (lane == L) {
        long long cum = incl - local;
#pragma unroll
        for (int k = 0; k < kEBins / 32; ++k) {
            if (sel.cls == kEBins && cum + c[k] >= A) {
                sel.cls = lane * (kEBins / 32) + k;
                sel.quota = (int)(A - cum);
            }
            cum += c[k];
        }
    }
    sel.cls = __shfl_sync(0xFFFFFFFFu, sel.cls, L);
    sel.quota = __shfl_sync(0xFFFFFFFFu, sel.quota, L);
    return sel;
}

// shared-memory records of the tracks that interact in one chunk, sorted by
// model (structure of arrays)
template <typename R, int BS>
struct Staging {
    double x[3][BS];
    R u[3][BS];
    R T[BS];
    uint64_t uid[BS];
    double dep[BS];
    long long src[BS];
    uint32_t ev[BS];
    uint32_t step[BS];
    uint32_t tv[BS];
    unsigned char model[BS];
    int count[kNumModels];
    int offset[kNumModels + 1];
};


// One step-loop iteration over both particle queues of side `side`.
// Counter slots: cin = this step's input counts, chunk dispenser and
// growth-token tally; cout = output counts (zero on entry); cclr = slot
// cleared for the next step (it held the previous step's input).
//
// Capacity: each input track owns one output slot (its survivor, or its
// copy when it is deferred).  A step never makes more than two outputs, so
// only a step with two outputs needs one of the Q - n spare slots: it takes
// a growth token first, and without one the step is discarded and the track
// is copied unchanged (its step counter, hence its random stream, is kept).
// Only interactions make two outputs.  When 2n <= Q every step fits and no
// token is counted.
template <typename R, int BS, int G, bool X>
__device__ __forceinline__ void step_body(const Params<R>& p, int side, int cin, int cout, int cclr, int& s_chunk,
                                          Staging<R, BS>& sg)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        p.cnt[cclr] = Counters{};
    }
    const Tracks<R> qi = p.q[side];
    const Tracks<R> qo = p.q[side ^ 1];
    const int nG = p.cnt[cin].n[0];
    const int nC = p.cnt[cin].n[1];
    const long long Q = p.Q;
    const long long ntot = (long long)nG + nC;
    const long long spare = Q - ntot;
    const bool unlimited = 2 * ntot <= Q;
    const int bs = BS;
    const int chunksG = (nG + bs - 1) / bs;
    const int chunksC = (nC + bs - 1) / bs;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const unsigned lanes_below = (1u << lane) - 1u;
    Counters* const co = &p.cnt[cout];

    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(&p.cnt[cin].work, 1);
        if (tid < kNumModels) sg.count[tid] = 0;
        __syncthreads();
        const int chunk = s_chunk;
        if (chunk >= chunksG + chunksC) break;
        const bool photon_chunk = chunk < chunksG;
        const long long i = photon_chunk ? (long long)chunk * bs + tid : (long long)(chunk - chunksG) * bs + tid;
        const long long n_here = photon_chunk ? nG : nC;
        const bool active = i < n_here;
        const long long src = photon_chunk ? i : Q - nC + i;

        // ---- phase A: own track
        TrackReg<R> t;
        Effects fx;
        StepOut<R> o;
        o.n = 0;
        int model = kNoInteraction;
        int rank = 0;
        int substeps = 0;
        if (active) {
            load_track(qi, src, t);
            bool alive;
            model = transport_part<G, X>(p, t, fx, alive);
            substeps = fx.substeps;
            if (model == kNoInteraction) {
                finish_step(p, t, alive, fx, o);
                apply_effects(p, t.ev, t.type, t.step, fx);
            } else {
                rank = atomicAdd(&sg.count[model], 1);
            }
        }
        count_substeps(p, lane, substeps);
        {
            const unsigned ms = __ballot_sync(0xFFFFFFFFu, active);
            if (lane == 0 && ms) atomicAdd(&p.total_steps[0], (unsigned long long)__popc(ms));
        }
        emit<1>(p, qo, co, lane, o, t.x, t.ev, t.vol);
        __syncthreads();
        if (tid == 0) {
            int acc = 0;
            for (int m = 0; m < kNumModels; ++m) {
                sg.offset[m] = acc;
                acc += sg.count[m];
            }
            sg.offset[kNumModels] = acc;
        }
        __syncthreads();
        if (model != kNoInteraction) {
            const int k = sg.offset[model] + rank;
            sg.x[0][k] = t.x[0];
            sg.x[1][k] = t.x[1];
            sg.x[2][k] = t.x[2];
            sg.u[0][k] = t.u[0];
            sg.u[1][k] = t.u[1];
            sg.u[2][k] = t.u[2];
            sg.T[k] = t.T;
            sg.uid[k] = t.uid;
            sg.dep[k] = fx.dep;
            sg.src[k] = src;
            sg.ev[k] = t.ev;
            sg.step[k] = t.step;
            sg.tv[k] = pack_tv(t.type, t.vol);
            sg.model[k] = (unsigned char)model;
        }
        __syncthreads();

        // ---- phase B: sampled interactions, sorted by model
        const int n_int = sg.offset[kNumModels];
        bool mine = tid < n_int;
        o.n = 0;
        bool stepped = false;
        long long rsrc = 0;
        if (mine) {
            t.x[0] = sg.x[0][tid];
            t.x[1] = sg.x[1][tid];
            t.x[2] = sg.x[2][tid];
            t.u[0] = sg.u[0][tid];
            t.u[1] = sg.u[1][tid];
            t.u[2] = sg.u[2][tid];
            t.T = sg.T[tid];
            t.uid = sg.uid[tid];
            t.ev = sg.ev[tid];
            t.step = sg.step[tid];
            t.type = tv_type(sg.tv[tid]);
            t.vol = tv_vol(sg.tv[tid]);
            rsrc = sg.src[tid];
            fx.dep = sg.dep[tid];
            fx.esc = 0.0;
            fx.kill = 0.0;
            fx.col = score_col(p, t.vol, t.x[2]);
            fx.finished = false;
            fx.live_delta = 0;
            interaction_part<X>(p, t, (int)sg.model[tid], fx, o);
            stepped = true;
        }
        if (!unlimited) {
            const bool need = stepped && o.n == 2;
            const unsigned m = __ballot_sync(0xFFFFFFFFu, need);
            if (m) {
                const int k = __popc(m);
                const int leader = __ffs(m) - 1;
                int got = 0;
                if (lane == leader) {
                    int old = atomicAdd(&p.cnt[cin].used, k);
                    long long avail = spare - old;
                    got = avail <= 0 ? 0 : (avail >= k ? k : (int)avail);
                    if (got < k) atomicSub(&p.cnt[cin].used, k - got);
                }
                got = __shfl_sync(0xFFFFFFFFu, got, leader);
                if (need && __popc(m & lanes_below) >= got) {
                    // no room for the second output: discard the whole step
                    load_track(qi, rsrc, t);
                    copy_out(t, o);
                    stepped = false;
                }
            }
        }
        if (stepped) apply_effects(p, t.ev, t.type, t.step, fx);
        {
            const unsigned md = __ballot_sync(0xFFFFFFFFu, mine && !stepped);
            if (lane == 0 && md) {
                atomicAdd(&p.total_steps[0], -(unsigned long long)__popc(md));
                atomicAdd(&p.total_steps[1], (unsigned long long)__popc(md));
            }
        }
        emit<2>(p, qo, co, lane, o, t.x, t.ev, t.vol);
        __syncthreads();
    }
}

template <typename R, int BS, int G, bool X>
__global__ void __launch_bounds__(BS, 512 / BS) k_step(Params<R> p, int side, int cin, int cout, int cclr)
{
    __shared__ int s_chunk;
    __shared__ Staging<R, BS> sg;
    step_body<R, BS, G, X>(p, side, cin, cout, cclr, s_chunk, sg);
}

// Grid-wide barrier of a persistent kernel whose blocks are all resident
// (cooperative launch): every block's thread 0 arrives on a counter, the
// last one resets it and advances the generation, the others wait for the
// generation to change.  The wait is bounded: after limit_cycles SM clock
// cycles (or once another block has given up) the block sets
// kStatusTimeout in the status word and returns false, so that the kernel
// ends and the host reports EMT_ERR_TIMEOUT instead of spinning forever.
__device__ __forceinline__ bool grid_barrier(GridSync* gs, unsigned blocks, long long limit_cycles, int* status)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* gen = &gs->gen;
        volatile int* vstatus = status;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(&gs->count, 1u) + 1u == blocks) {
            gs->count = 0u;
            __threadfence();
            atomicAdd(&gs->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if ((*vstatus & kStatusTimeout) || clock64() - t0 > limit_cycles) {
                    atomicOr(status, kStatusTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Persistent step loop: up to max_steps steps of the fused schedule in one
// launch, from global iteration it0 (its counter slots and ping-pong side),
// with a grid barrier after each step; the launch ends early when no track
// is left.  Removes the launch gap between steps (the paper's many
// synchronization points per step, Sec. 3.2) where a step is short: the
// tail of a run, one event at a time, a served stream at a low rate.
// gs->iters receives the number of steps run.
template <typename R, int BS, int G, bool X>
__global__ void __launch_bounds__(BS, 512 / BS)
    k_persist(Params<R> p, long long it0, int max_steps, GridSync* gs, long long limit_cycles)
{
    __shared__ int s_chunk;
    __shared__ Staging<R, BS> sg;
    __shared__ int s_go;
    int done = 0;
    while (done < max_steps) {
        const long long it = it0 + done;
        const int side = (int)(it & 1), cin = (int)(it % 3), cout = (int)((it + 1) % 3), cclr = (int)((it + 2) % 3);
        step_body<R, BS, G, X>(p, side, cin, cout, cclr, s_chunk, sg);
        ++done;
        if (!grid_barrier(gs, gridDim.x, limit_cycles, p.status)) return;
        if (threadIdx.x == 0) s_go = p.cnt[cout].n[0] + p.cnt[cout].n[1] > 0;
        __syncthreads();
        const bool go = s_go != 0;
        __syncthreads();
        if (!go) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) gs->iters = (unsigned)done;
}


// Admit primaries (structure of arrays, device memory) into side `side`,
// appending after the tracks already counted in slot `cs`.  Primaries
// below their cut deposit at once; outside the world they escape.
template <typename R>
__global__ void k_admit(Params<R> p, int side, int cs, int n, const int32_t* ev, const int32_t* type,
                        const double* T, const double* pos, const double* dir, const uint32_t* slot_of_event,
                        const uint32_t* uid_of)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool keep = false;
    TrackReg<R> t;
    if (i < n) {
        t.ev = slot_of_event[ev[i]];
        t.type = type[i];
        t.T = R(T[i]);
        t.x[0] = pos[3 * i + 0];
        t.x[1] = pos[3 * i + 1];
        t.x[2] = pos[3 * i + 2];
        t.u[0] = R(dir[3 * i + 0]);
        t.u[1] = R(dir[3 * i + 1]);
        t.u[2] = R(dir[3 * i + 2]);
        t.uid = uid_of[i];
        t.step = 0;
        const int vol = locate_volume(p, t.x);
        t.vol = vol;
        double E = (double)T[i] + rest_energy(t.type);
        if (t.type < 0 || t.type > 2) {
            atomicOr(p.status, kStatusBadTrack);
        } else {
            atomicAdd(&p.ledger[3 * (size_t)t.ev + 2], E);
            if (vol == kVolOut) {
                atomicAdd(&p.ledger[3 * (size_t)t.ev + 0], E);
            } else if (T[i] < p.cut[t.type]) {
                deposit_now(p, t.ev, score_col(p, vol, t.x[2]), E);
            } else {
                keep = true;
                atomicAdd(&p.live[t.ev], 1);
                if (p.max_active > 0) atomicAdd(&p.ehist[(size_t)cs * kEBins + energy_class(est_f(t.T))], 1u);
            }
        }
    }
    unsigned mG = __ballot_sync(0xFFFFFFFFu, keep && t.type == 0);
    unsigned mC = __ballot_sync(0xFFFFFFFFu, keep && t.type != 0);
    int baseG = 0, baseC = 0;
    if (lane == 0) {
        if (mG) baseG = atomicAdd(&p.cnt[cs].n[0], __popc(mG));
        if (mC) baseC = atomicAdd(&p.cnt[cs].n[1], __popc(mC));
    }
    baseG = __shfl_sync(0xFFFFFFFFu, baseG, 0);
    baseC = __shfl_sync(0xFFFFFFFFu, baseC, 0);
    if (keep) {
        unsigned below = (1u << lane) - 1u;
        long long dst = t.type == 0 ? (long long)baseG + __popc(mG & below)
                                    : p.Q - 1 - ((long long)baseC + __popc(mC & below));
        if (dst < 0 || dst >= p.Q) {
            atomicOr(p.status, kStatusQueueOverflow);
        } else {
            store_track(p.q[side], dst, t.x, t.u, t.T, t.uid, t.ev, t.step, t.type, t.vol);
        }
    }
}

// Host spill: append n tracks of the spill buffer (records 0..n-1, moved
// back from host memory) to side `side`, counted in slot `cs`.  Their
// events still count them as alive.
template <typename R>
__global__ void k_unspill(Params<R> p, int side, int cs, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    TrackReg<R> t;
    const bool have = i < n;
    if (have) load_track(p.spill, i, t);
    const unsigned mG = __ballot_sync(0xFFFFFFFFu, have && t.type == 0);
    const unsigned mC = __ballot_sync(0xFFFFFFFFu, have && t.type != 0);
    int baseG = 0, baseC = 0;
    if (lane == 0) {
        if (mG) baseG = atomicAdd(&p.cnt[cs].n[0], __popc(mG));
        if (mC) baseC = atomicAdd(&p.cnt[cs].n[1], __popc(mC));
    }
    baseG = __shfl_sync(0xFFFFFFFFu, baseG, 0);
    baseC = __shfl_sync(0xFFFFFFFFu, baseC, 0);
    if (!have) return;
    const unsigned below = (1u << lane) - 1u;
    const long long dst = t.type == 0 ? (long long)baseG + __popc(mG & below)
                                      : p.Q - 1 - ((long long)baseC + __popc(mC & below));
    if (dst < 0 || dst >= p.Q) {
        atomicOr(p.status, kStatusQueueOverflow);
        return;
    }
    store_track(p.q[side], dst, t.x, t.u, t.T, t.uid, t.ev, t.step, t.type, t.vol);
    atomicAdd(&p.ehist[(size_t)cs * kEBins + energy_class(est_f(t.T))], 1u);
}

// Diagnostics: write explicit track records into side `side`.
template <typename R>
__global__ void k_set_tracks(Params<R> p, int side, int cs, int n, const double* rec, const uint64_t* uid,
                             const int32_t* slot)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* r = rec + 10 * (size_t)i;
    int type = (int)r[0];
    double x[3] = {r[2], r[3], r[4]};
    R u[3] = {R(r[5]), R(r[6]), R(r[7])};
    long long dst;
    if (type == 0)
        dst = atomicAdd(&p.cnt[cs].n[0], 1);
    else
        dst = p.Q - 1 - atomicAdd(&p.cnt[cs].n[1], 1);
    if (dst < 0 || dst >= p.Q) {
        atomicOr(p.status, kStatusQueueOverflow);
        return;
    }
    atomicAdd(&p.live[slot[i]], 1);
    if (p.max_active > 0) atomicAdd(&p.ehist[(size_t)cs * kEBins + energy_class(est_f(R(r[1])))], 1u);
    store_track(p.q[side], dst, x, u, R(r[1]), uid[i], (uint32_t)slot[i], (uint32_t)r[9], type, (int)r[8]);
}

template <typename R>
__global__ void k_get_tracks(Params<R> p, int side, int nG, int nC, double* rec, uint64_t* uid, int32_t* slot)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nG + nC) return;
    long long src = i < nG ? i : p.Q - nC + (i - nG);
    TrackReg<R> t;
    load_track(p.q[side], src, t);
    double* r = rec + 10 * (size_t)i;
    r[0] = t.type;
    r[1] = (double)t.T;
    r[2] = t.x[0];
    r[3] = t.x[1];
    r[4] = t.x[2];
    r[5] = (double)t.u[0];
    r[6] = (double)t.u[1];
    r[7] = (double)t.u[2];
    r[8] = t.vol;
    r[9] = t.step;
    uid[i] = t.uid;
    slot[i] = (int32_t)t.ev;
}

}  // namespace emt
