// emt_split.cuh -- the split schedule of one step: a transport kernel and
// an interaction kernel per step-loop iteration.
//
// The fused kernel (emt_step.cuh) regroups the interacting tracks of each
// chunk inside its block, which leaves most warps of the block waiting at
// a barrier while a few run the samplers.  Here the transport kernel runs
// phase A for every track and appends the tracks that interact to a global
// queue (warp-aggregated, one atomic per warp); the interaction kernel then
// takes the queue in full chunks, counting-sorts each chunk by model in
// shared memory and samples with every lane busy.  The cost is one more
// write and read of the interacting tracks' state (a few percent of the
// step's track-state traffic); the results are the same as the fused
// schedule's (same arithmetic, same random streams).
#pragma once

#include "emt_step.cuh"

namespace emt {

__device__ __forceinline__ uint32_t pack_tvm(int type, int vol, int model)
{
    return (uint32_t)type | ((uint32_t)(vol + 2) << 8) | ((uint32_t)model << 24);
}

// Track selection (max_active > 0): the tracks that do not fit the step's
// budget are held, copied unchanged with their step counter, so they draw
// the same random numbers when they do step and no result depends on the
// policy; both kernels count their outputs' energy classes for the next
// step's selection.
// Resident threads per SM the transport kernel is compiled for (its
// register budget), measured on GB300.  FP64: 512 (128 registers, almost no
// spills).  In a field the RK4 substeps keep many doubles live; at 768
// threads (80 registers) their spills share the FP64 unit's issue queue,
// and the field transport runs 13% slower.  Without a field 768 was 1% faster,
// but there the pipelined schedule is used.  Mixed precision: 640 (768
// measured 14% slower in the field, 2% faster on the cylinder problem).
template <typename R>
constexpr int transport_threads_per_sm()
{
    return sizeof(R) == 8 ? 512 : 640;
}

// Phase A of one track in the transport kernel (every lane of the warp
// calls it; `active` lanes hold a track in t, `held` ones are copied
// unchanged): transport, survivor output, and the queueing of an
// interacting track (into iq, counted in *n_iq) for the interaction phase.
// count_queued: a queued track's step is counted now (split schedule) or
// when its interaction is committed (pipelined schedule).
template <int G, bool X, typename R>
__device__ __forceinline__ void transport_lane(const Params<R>& p, const Tracks<R>& qo, Counters* co,
                                               const InterQueue<R>& iq, int* n_iq, bool count_queued, int lane,
                                               TrackReg<R>& t, bool active, bool held, long long src, unsigned* eh)
{
    const unsigned lanes_below = (1u << lane) - 1u;
    Effects fx;
    StepOut<R> o;
    o.n = 0;
    int model = kNoInteraction;
    int substeps = 0;
    if (held) {
        copy_out(t, o);
    } else if (active) {
        bool alive;
        model = transport_part<G, X>(p, t, fx, alive);
        substeps = fx.substeps;
        if (model == kNoInteraction) {
            finish_step(p, t, alive, fx, o);
            apply_effects(p, t.ev, t.type, t.step, fx);
        }
    }
    count_substeps(p, lane, substeps);
    {
        const unsigned ms = __ballot_sync(0xFFFFFFFFu, active && !held && (count_queued || model == kNoInteraction));
        if (lane == 0 && ms) atomicAdd(&p.total_steps[0], (unsigned long long)__popc(ms));
    }
    emit<1>(p, qo, co, lane, o, t.x, t.ev, t.vol, eh);
    // queue the interacting tracks
    const bool need = model != kNoInteraction;
    const unsigned m = __ballot_sync(0xFFFFFFFFu, need);
    if (m) {
        int base = 0;
        if (lane == 0) base = atomicAdd(n_iq, __popc(m));
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (need) {
            const long long k = (long long)base + __popc(m & lanes_below);
            if (k < p.Q) {
                iq.x[k] = t.x[0];
                iq.y[k] = t.x[1];
                iq.z[k] = t.x[2];
                iq.ux[k] = t.u[0];
                iq.uy[k] = t.u[1];
                iq.uz[k] = t.u[2];
                iq.T[k] = t.T;
                iq.uid[k] = t.uid;
                iq.dep[k] = fx.dep;
                iq.ev[k] = t.ev;
                iq.step[k] = t.step;
                iq.tv[k] = pack_tvm(t.type, t.vol, model);
                iq.src[k] = (uint32_t)src;
            } else {
                atomicOr(p.status, kStatusQueueOverflow);
            }
        }
    }
}

// The charged tracks of a step in a field, sorted by expected cost (a
// counting sort by scheduling class, two launches before the transport
// kernel): k_sort_keys estimates each track's RK4 substep count and counts
// the classes; k_sort_order writes the order, most expensive class first.
// The transport kernel then takes the charged tracks in that order, a warp
// at a time: warps run lanes of similar substep counts (instead of a random
// mix, whose slowest lane sets the warp's time), the expensive warps start
// first and the cheap ones fill the end of the launch.  The order within a
// class is arbitrary; results do not depend on it.
template <typename R>
__global__ void __launch_bounds__(256) k_sort_keys(Params<R> p, int side, int cin)
{
    __shared__ int h[kSortKeys];
    if (threadIdx.x < kSortKeys) h[threadIdx.x] = 0;
    __syncthreads();
    const int nC = p.cnt[cin].n[1];
    const Tracks<R> qi = p.q[side];
    const long long base = p.Q - nC;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nC;
         i += (long long)gridDim.x * blockDim.x) {
        TrackReg<R> t;
        t.T = qi.T[base + i];
        t.uid = qi.uid[base + i];
        t.ev = qi.ev[base + i];
        t.step = qi.step[base + i];
        const uint32_t tv = qi.tv[base + i];
        t.type = tv_type(tv);
        t.vol = tv_vol(tv);
        t.x[2] = qi.z[base + i];
        t.u[2] = qi.uz[base + i];
        const int cls = substep_class(field_substeps_estimate(p, t));
        p.skey[i] = (uint8_t)cls;
        atomicAdd(&h[cls], 1);
    }
    __syncthreads();
    if (threadIdx.x < kSortKeys && h[threadIdx.x]) atomicAdd(&p.cnt[cin].kbin[threadIdx.x], h[threadIdx.x]);
}

template <typename R>
__global__ void __launch_bounds__(256) k_sort_order(Params<R> p, int cin)
{
    __shared__ int off[kSortKeys], cnt[kSortKeys], base[kSortKeys];
    const int tid = threadIdx.x;
    const int nC = p.cnt[cin].n[1];
    if (tid < 32) {
        // first place of each class: exclusive prefix sum of the counts
        const int c = tid < kSortKeys ? p.cnt[cin].kbin[tid] : 0;
        int incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
            if (tid >= d) incl += y;
        }
        if (tid < kSortKeys) off[tid] = incl - c;
    }
    for (long long first = (long long)blockIdx.x * blockDim.x; first < nC; first += (long long)gridDim.x * blockDim.x) {
        if (tid < kSortKeys) cnt[tid] = 0;
        __syncthreads();
        const long long i = first + tid;
        int key = -1, rank = 0;
        if (i < nC) {
            key = p.skey[i];
            rank = atomicAdd(&cnt[key], 1);
        }
        __syncthreads();
        if (tid < kSortKeys && cnt[tid]) base[tid] = atomicAdd(&p.cnt[cin].kcur[tid], cnt[tid]);
        __syncthreads();
        if (key >= 0) p.sperm[off[key] + base[key] + rank] = (uint32_t)i;
        __syncthreads();
    }
}

template <typename R, int BS, int G, bool S, bool X>
__global__ void __launch_bounds__(BS, transport_threads_per_sm<R>() / BS)
    k_transport(Params<R> p, int side, int cin, int cout, int cclr)
{
    __shared__ int s_chunk;
    __shared__ unsigned s_eh[S ? kEBins : 1];
    __shared__ Selection s_sel, s_spill;
    constexpr bool select = S;
    if (blockIdx.x == 0 && threadIdx.x == 0) p.cnt[cclr] = Counters{};
    const Tracks<R> qi = p.q[side];
    const Tracks<R> qo = p.q[side ^ 1];
    const int nG = p.cnt[cin].n[0];
    const int nC = p.cnt[cin].n[1];
    const long long Q = p.Q;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const unsigned lanes_below = (1u << lane) - 1u;
    Counters* const co = &p.cnt[cout];
    // In a field the charged tracks (tens of RK4 substeps per step) are
    // handed out before the photons, so that the cheap photon work fills
    // the end of the launch instead of the expensive charged work.
    const bool charged_first = p.has_field != 0;

    if constexpr (!select) {
        // Chunks of one warp, taken by each warp on its own (no block
        // barrier: a warp never waits for the slowest warp of its block).
        // In a field the charged tracks are taken in the order of
        // k_sort_order (most expensive first).
        const int chunksG = (nG + 31) >> 5;
        const int chunksC = (nC + 31) >> 5;
        const bool sorted = p.has_field != 0;
        for (;;) {
            int chunk = 0;
            if (lane == 0) chunk = atomicAdd(&p.cnt[cin].work, 1);
            chunk = __shfl_sync(0xFFFFFFFFu, chunk, 0);
            if (chunk >= chunksG + chunksC) break;
            const bool photon_chunk = charged_first ? chunk >= chunksC : chunk < chunksG;
            const int local = photon_chunk ? (charged_first ? chunk - chunksC : chunk)
                                           : (charged_first ? chunk : chunk - chunksG);
            long long i = (long long)local * 32 + lane;
            const bool active = i < (photon_chunk ? nG : nC);
            if (sorted && !photon_chunk && active) i = p.sperm[i];
            const long long src = photon_chunk ? i : Q - nC + i;
            TrackReg<R> t;
            if (active) load_track(qi, src, t);
            transport_lane<G, X>(p, qo, co, p.iq, &p.cnt[cin].n_int, true, lane, t, active, false, src, nullptr);
        }
        return;
    }

    // track selection: chunks of a block (the selection is block-wide)
    if constexpr (select) {
        for (int b = threadIdx.x; b < kEBins; b += BS) {
            s_eh[b] = 0u;
            if (blockIdx.x == 0) p.ehist[(size_t)cclr * kEBins + b] = 0u;
        }
        if (threadIdx.x < 32) {
            Selection sl, sp;
            sl.cls = sp.cls = kEBins;
            sl.quota = sp.quota = 0;
            if (p.select_policy == kSelectLowEnergy) {
                sl = select_threshold(p, cin, threadIdx.x, p.max_active);
                if (p.spill_above > 0) sp = select_threshold(p, cin, threadIdx.x, p.spill_above);
            }
            if (threadIdx.x == 0) {
                s_sel = sl;
                s_spill = sp;
                if (blockIdx.x == 0) p.spill_ticket[cclr] = 0;
            }
        }
        __syncthreads();
    }
    const int chunksG = (nG + BS - 1) / BS;
    const int chunksC = (nC + BS - 1) / BS;
    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(&p.cnt[cin].work, 1);
        __syncthreads();
        const int chunk = s_chunk;
        __syncthreads();
        if (chunk >= chunksG + chunksC) break;
        const bool photon_chunk = charged_first ? chunk >= chunksC : chunk < chunksG;
        const int local = photon_chunk ? (charged_first ? chunk - chunksC : chunk)
                                       : (charged_first ? chunk : chunk - chunksG);
        const long long i = (long long)local * BS + tid;
        const long long n_here = photon_chunk ? nG : nC;
        bool active = i < n_here;
        const long long src = photon_chunk ? i : Q - nC + i;

        TrackReg<R> t;
        bool held = false;
        if (active) load_track(qi, src, t);
        if constexpr (select) {
            if (p.select_policy == kSelectOrder) {
                held = active && (photon_chunk ? i : nG + i) >= p.max_active;
            } else {
                const int cls = active ? energy_class(est_f(t.T)) : kEBins + 1;
                held = cls > s_sel.cls && cls <= kEBins;
                int t1 = -1, t2 = -1;  // tickets in the boundary classes
                const bool edge = cls == s_sel.cls;
                const unsigned me = __ballot_sync(0xFFFFFFFFu, edge);
                if (me) {
                    int base = 0;
                    if (lane == __ffs(me) - 1) base = atomicAdd(&p.cnt[cin].ticket, __popc(me));
                    base = __shfl_sync(0xFFFFFFFFu, base, __ffs(me) - 1);
                    t1 = base + __popc(me & lanes_below);
                    if (edge) held = t1 >= s_sel.quota;
                }
                if (p.spill_above > 0) {
                    // the held tracks above the spill_above lowest-energy ones
                    // leave the device
                    const bool edge2 = cls == s_spill.cls && s_spill.cls != s_sel.cls;
                    const unsigned m2 = __ballot_sync(0xFFFFFFFFu, edge2);
                    if (m2) {
                        int base = 0;
                        if (lane == __ffs(m2) - 1) base = atomicAdd(&p.spill_ticket[cin], __popc(m2));
                        base = __shfl_sync(0xFFFFFFFFu, base, __ffs(m2) - 1);
                        t2 = base + __popc(m2 & lanes_below);
                    }
                    if (s_spill.cls == s_sel.cls) t2 = t1;
                    const bool go = held && (cls > s_spill.cls || (cls == s_spill.cls && t2 >= s_spill.quota));
                    const unsigned mg = __ballot_sync(0xFFFFFFFFu, go);
                    if (mg) {
                        int base = 0;
                        if (lane == 0) base = atomicAdd(&p.cnt[cin].spilled, __popc(mg));
                        base = __shfl_sync(0xFFFFFFFFu, base, 0);
                        const long long k = (long long)base + __popc(mg & lanes_below);
                        if (go && k < p.spill_cap) {
                            store_track(p.spill, k, t.x, t.u, t.T, t.uid, t.ev, t.step, t.type, t.vol);
                            held = false;  // neither stepped nor kept on the device
                            active = false;
                        }
                    }
                }
            }
            const unsigned mh = __ballot_sync(0xFFFFFFFFu, held);
            if (lane == 0 && mh) atomicAdd(&p.total_steps[2], (unsigned long long)__popc(mh));
        }
        transport_lane<G, X>(p, qo, co, p.iq, &p.cnt[cin].n_int, true, lane, t, active, held, src, s_eh);
    }
    if constexpr (select) {
        __syncthreads();
        for (int b = threadIdx.x; b < kEBins; b += BS)
            if (s_eh[b]) atomicAdd(&p.ehist[(size_t)cout * kEBins + b], s_eh[b]);
    }
}

// Queue records per thread in one chunk of the interaction kernel: a block
// counting-sorts kInteractRecords * BS records by model and its warps take
// them in sorted order, kInteractRecords rounds of 32 each; larger sorted
// chunks give warps of fewer models.
constexpr int kInteractRecords = 2;

// copy queue record r of `from` to record k of `to`
template <typename R>
__device__ __forceinline__ void copy_record(const InterQueue<R>& from, long long r, const InterQueue<R>& to, long long k)
{
    to.x[k] = from.x[r];
    to.y[k] = from.y[r];
    to.z[k] = from.z[r];
    to.ux[k] = from.ux[r];
    to.uy[k] = from.uy[r];
    to.uz[k] = from.uz[r];
    to.T[k] = from.T[r];
    to.uid[k] = from.uid[r];
    to.dep[k] = from.dep[r];
    to.ev[k] = from.ev[r];
    to.step[k] = from.step[r];
    to.tv[k] = from.tv[r];
    to.src[k] = from.src[r];
}

// The interaction phase over the n_int records of queue iq: chunks of
// kInteractRecords * BS records, each counting-sorted by model in shared
// memory and sampled by the block's warps in sorted order.  A record whose
// step makes two outputs needs a growth token from the `spare` slots; a
// step without one is deferred: split schedule (kPipe false): the track is
// copied unchanged from the input buffer qi (it repeats the whole step);
// pipelined schedule: the record is queued again, unchanged, in qnext
// (counted in *n_next), and its interaction is sampled in the next
// iteration.  Either way it keeps its step counter, so no result changes.
// Every thread of the block calls it (barriers).
template <typename R, int BS, bool X, bool kPipe>
__device__ __forceinline__ void interact_chunks(const Params<R>& p, const Tracks<R>& qi, const Tracks<R>& qo,
                                                Counters* co, int cin, const InterQueue<R>& iq, int n_int,
                                                long long spare, bool unlimited, const InterQueue<R>& qnext,
                                                int* n_next, unsigned* eh, int& s_chunk, int* count, int* offset,
                                                unsigned short* perm)
{
    constexpr int CH = BS * kInteractRecords;
    const int chunks = (n_int + CH - 1) / CH;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const unsigned lanes_below = (1u << lane) - 1u;
    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(&p.cnt[cin].work_b, 1);
        if (tid < kNumModels) count[tid] = 0;
        __syncthreads();
        const int chunk = s_chunk;
        if (chunk >= chunks) break;
        const long long r0 = (long long)chunk * CH;
        const int n_here = (int)(n_int - r0 < CH ? n_int - r0 : CH);
        // counting sort of the chunk's records by model
        int model[kInteractRecords], rank[kInteractRecords];
#pragma unroll
        for (int j = 0; j < kInteractRecords; ++j) {
            const int idx = j * BS + tid;
            model[j] = -1;
            rank[j] = 0;
            if (idx < n_here) {
                model[j] = (int)(iq.tv[r0 + idx] >> 24);
                rank[j] = atomicAdd(&count[model[j]], 1);
            }
        }
        __syncthreads();
        if (tid == 0) {
            int acc = 0;
            for (int k = 0; k < kNumModels; ++k) {
                offset[k] = acc;
                acc += count[k];
            }
            offset[kNumModels] = acc;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kInteractRecords; ++j)
            if (model[j] >= 0) perm[offset[model[j]] + rank[j]] = (unsigned short)(j * BS + tid);
        __syncthreads();

        for (int round = 0; round < kInteractRecords; ++round) {
            const int pos = round * BS + tid;  // sorted position: a warp takes 32 consecutive ones
            const bool mine = pos < n_here;
            TrackReg<R> t;
            Effects fx;
            StepOut<R> o;
            o.n = 0;
            bool stepped = false;
            long long rsrc = 0;
            long long r = 0;
            if (mine) {
                r = r0 + perm[pos];
                const uint32_t tv = iq.tv[r];
                t.x[0] = iq.x[r];
                t.x[1] = iq.y[r];
                t.x[2] = iq.z[r];
                t.u[0] = iq.ux[r];
                t.u[1] = iq.uy[r];
                t.u[2] = iq.uz[r];
                t.T = iq.T[r];
                t.uid = iq.uid[r];
                t.ev = iq.ev[r];
                t.step = iq.step[r];
                t.type = (int)(tv & 0xFFu);
                t.vol = (int)((tv >> 8) & 0xFFFFu) - 2;
                rsrc = iq.src[r];
                fx.dep = iq.dep[r];
                fx.esc = 0.0;
                fx.kill = 0.0;
                fx.col = score_col(p, t.vol, t.x[2]);
                fx.finished = false;
                fx.live_delta = 0;
                interaction_part<X>(p, t, (int)(tv >> 24), fx, o);
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
                        // no room for the second output: discard the step
                        if constexpr (kPipe) {
                            o.n = 0;
                        } else {
                            load_track(qi, rsrc, t);
                            copy_out(t, o);
                        }
                        stepped = false;
                    }
                }
            }
            if (stepped) apply_effects(p, t.ev, t.type, t.step, fx);
            {
                const unsigned md = __ballot_sync(0xFFFFFFFFu, mine && !stepped);
                if constexpr (kPipe) {
                    // the step of an interacting track counts when it commits
                    const unsigned mc = __ballot_sync(0xFFFFFFFFu, mine && stepped);
                    if (lane == 0 && mc) atomicAdd(&p.total_steps[0], (unsigned long long)__popc(mc));
                    if (lane == 0 && md) atomicAdd(&p.total_steps[1], (unsigned long long)__popc(md));
                    if (md) {
                        int base = 0;
                        if (lane == 0) base = atomicAdd(n_next, __popc(md));
                        base = __shfl_sync(0xFFFFFFFFu, base, 0);
                        if (mine && !stepped) {
                            const long long k = (long long)base + __popc(md & lanes_below);
                            if (k < p.Q)
                                copy_record(iq, r, qnext, k);
                            else
                                atomicOr(p.status, kStatusQueueOverflow);
                        }
                    }
                } else {
                    if (lane == 0 && md) {
                        atomicAdd(&p.total_steps[0], -(unsigned long long)__popc(md));
                        atomicAdd(&p.total_steps[1], (unsigned long long)__popc(md));
                    }
                }
            }
            emit<2>(p, qo, co, lane, o, t.x, t.ev, t.vol, eh);
        }
        __syncthreads();
    }
}

template <typename R, int BS, bool S, bool X>
__global__ void __launch_bounds__(BS, 512 / BS) k_interact(Params<R> p, int side, int cin, int cout)
{
    constexpr int CH = BS * kInteractRecords;
    __shared__ int s_chunk;
    __shared__ int count[kNumModels];
    __shared__ int offset[kNumModels + 1];
    __shared__ unsigned short perm[CH];
    __shared__ unsigned s_eh[S ? kEBins : 1];
    constexpr bool select = S;
    if constexpr (select) {
        for (int b = threadIdx.x; b < kEBins; b += BS) s_eh[b] = 0u;
        __syncthreads();
    }
    const long long ntot = (long long)p.cnt[cin].n[0] + p.cnt[cin].n[1];
    interact_chunks<R, BS, X, false>(p, p.q[side], p.q[side ^ 1], &p.cnt[cout], cin, p.iq, p.cnt[cin].n_int,
                                     p.Q - ntot, 2 * ntot <= p.Q, p.iq, nullptr, select ? s_eh : nullptr, s_chunk,
                                     count, offset, perm);
    if constexpr (select) {
        for (int b = threadIdx.x; b < kEBins; b += BS)
            if (s_eh[b]) atomicAdd(&p.ehist[(size_t)cout * kEBins + b], s_eh[b]);
    }
}

// Resident threads per SM of the pipelined kernel (its register budget).
// FP64: 512 (128 registers, the interaction phase without spills); mixed
// precision: 768 (about 80 registers, little spilled), whose extra
// resident warps hide more of the transport phase's latency (+3% on the
// calorimeter against 512; the FP64 kernel at 768 spills ~500 bytes a
// thread and gains nothing).
template <typename R>
constexpr int pipe_threads_per_sm()
{
    return sizeof(R) == 8 ? 512 : 768;
}

// Pipelined schedule: one kernel per step-loop iteration.  Its blocks
// first sample the interactions queued by the previous iteration (queue
// iq_side[side ^ 1], block-level chunks sorted by model), then transport
// this iteration's tracks a warp-sized chunk at a time, queueing the
// tracks that interact in iq_side[side] (counted in the output counter
// slot, so the next iteration finds them).  Transport and interaction work
// of the same launch overlap on the GPU instead of running as two launches
// one after the other; an interacting track's step simply completes one
// iteration later.  Each input track and each queued record owns one output
// slot; a record with two outputs takes a growth token from the rest.
template <typename R, int BS, int G, bool X>
__global__ void __launch_bounds__(BS, pipe_threads_per_sm<R>() / BS)
    k_pipe(Params<R> p, int side, int cin, int cout, int cclr)
{
    constexpr int CH = BS * kInteractRecords;
    __shared__ int s_chunk;
    __shared__ int count[kNumModels];
    __shared__ int offset[kNumModels + 1];
    __shared__ unsigned short perm[CH];
    if (blockIdx.x == 0 && threadIdx.x == 0) p.cnt[cclr] = Counters{};
    const Tracks<R> qi = p.q[side];
    const Tracks<R> qo = p.q[side ^ 1];
    const InterQueue<R> q_prev = side ? p.iq : p.iq_alt;
    const InterQueue<R> q_next = side ? p.iq_alt : p.iq;
    int* const n_next = &p.cnt[cout].n_int;
    const int nG = p.cnt[cin].n[0];
    const int nC = p.cnt[cin].n[1];
    const int n_prev = p.cnt[cin].n_int;
    const long long Q = p.Q;
    const long long ntot = (long long)nG + nC + n_prev;
    Counters* const co = &p.cnt[cout];

    // interactions of the previous iteration
    interact_chunks<R, BS, X, true>(p, qi, qo, co, cin, q_prev, n_prev, Q - ntot, 2 * ntot <= Q, q_next, n_next,
                                    nullptr, s_chunk, count, offset, perm);

    // transport of this iteration's tracks (charged first in a field, in
    // the order of k_sort_order)
    const int lane = threadIdx.x & 31;
    const int chunksG = (nG + 31) >> 5;
    const int chunksC = (nC + 31) >> 5;
    const bool charged_first = p.has_field != 0;
    for (;;) {
        int chunk = 0;
        if (lane == 0) chunk = atomicAdd(&p.cnt[cin].work, 1);
        chunk = __shfl_sync(0xFFFFFFFFu, chunk, 0);
        if (chunk >= chunksG + chunksC) break;
        const bool photon_chunk = charged_first ? chunk >= chunksC : chunk < chunksG;
        const int local = photon_chunk ? (charged_first ? chunk - chunksC : chunk)
                                       : (charged_first ? chunk : chunk - chunksG);
        long long i = (long long)local * 32 + lane;
        const bool active = i < (photon_chunk ? nG : nC);
        if (charged_first && !photon_chunk && active) i = p.sperm[i];
        const long long src = photon_chunk ? i : Q - nC + i;
        TrackReg<R> t;
        if (active) load_track(qi, src, t);
        transport_lane<G, X>(p, qo, co, q_next, n_next, false, lane, t, active, false, src, nullptr);
    }
}

}  // namespace emt
