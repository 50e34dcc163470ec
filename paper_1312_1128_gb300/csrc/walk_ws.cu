// walk_ws.cu -- the tree walk with producer and consumer warps (Sec. 3.2 walk,
// Sec. 3.3 ray-parallel evaluation).
//
// The walk kernel alternates, in every warp, a latency-bound phase (popping
// boxes, the MAC, scanning big lists: dependent global loads) with an
// arithmetic-bound phase (evaluating a full buffer for the group's rays).  Here
// the two phases run in different warps of a pair: the producer walks the tree
// for a group and fills one of two shared-memory slots (far cells, leaf
// particles, big-list entries); when any buffer of the slot is full, or the
// group is done, it hands the slot to the consumer and continues in the other
// slot.  The consumer holds the group's rays and evaluates every slot it
// receives; at the group's last slot it adds the analytic halos and stores the
// totals.  Each hand-over is an mbarrier phase (all 32 lanes arrive; every
// lane acquires before reading), and every wait is bounded (the tree's wait
// limit, about 2 s of SM clock by default): a wait that gives up latches
// DERR_WAIT_TIMEOUT and both warps return -- the consumer at once, the
// producer at its next hand-over, which then waits for nobody.
#include "walk_dev.cuh"

namespace lens {

constexpr int kWsPairs = 4;                  // producers (one per team) per block
// A team is one producer warp and CONS consumer warps: CONS = 1 (pairs; the
// consumer holds the whole group, R rays per lane) or CONS = 2 (trios: a
// 64-ray group split between two consumers, 32 rays each).  The block's
// warps are the producers (warpgroup 0) and then each consumer rank's
// warpgroup.
template <int CONS> struct WsShape {
    static constexpr int kThreads = (1 + CONS) * kWsPairs * 32;
    static constexpr int kBlocksPerSm = CONS == 1 ? 3 : 2;
    // Registers per thread: the kernel is compiled for kLaunchRegs; the
    // producer warpgroup then gives registers back and each consumer
    // warpgroup takes them: 128 (kProdRegs + CONS kConsRegs) equals the
    // block's kThreads x kLaunchRegs, checked on the host before every launch.
    static constexpr int kLaunchRegs = 80, kProdRegs = 64, kConsRegs = CONS == 1 ? 96 : 88;
    static_assert(kProdRegs + CONS * kConsRegs == (1 + CONS) * kLaunchRegs, "register split must use the launch budget");
};
enum : int { kWsLast = 1, kWsStop = 2 };

template <int KIND, typename T> struct WsSlot {
    WalkBuf<KIND, T> buf;
    int nf, nn, nb;  // entries in the far, near and big buffers
    int g;           // group the entries belong to
    int flags;       // kWsLast: the group's last slot; kWsStop: no more groups
};

template <int KIND, typename T, int CONS> struct WsPair {
    WsSlot<KIND, T> slot[2];
    unsigned long long full[2], empty[2];  // mbarriers: 32 and 32 CONS arrivals
    WalkRanges rng;                        // the producer's list ranges
    WalkTot<T> tot[CONS];                  // each consumer's compensated totals
};

LENS_DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

LENS_DEV void mbar_init(unsigned long long* b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

LENS_DEV void mbar_arrive(unsigned long long* b)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b))
                 : "memory");
}

LENS_DEV bool mbar_try_wait(unsigned long long* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait, warp-uniformly, for the completion of the barrier phase of the given
// parity: every lane polls (each acquiring the phase for itself) for at most
// `limit` SM clock cycles.  Returns false (error latched) if any lane gave up.
LENS_DEV bool mbar_wait(unsigned long long* b, uint32_t parity, uint32_t* err, long long limit)
{
    bool ok = true;
    const long long t0 = clock64();
    while (!mbar_try_wait(b, parity)) {
        if (clock64() - t0 > limit) {
            ok = false;
            break;
        }
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && (threadIdx.x & 31) == 0) atomicOr(err, DERR_WAIT_TIMEOUT);
    return ok;
}

// The producer's context: the traversal and the appends of walk_dev.cuh write
// into the current slot; a full buffer hands the slot over.
template <int KIND, typename T, int CONS> struct WsProducer {
    using value_type = T;
    using Buf = WalkBuf<KIND, T>;
    static constexpr int kKind = KIND;
    static constexpr int kNear = Buf::kNear, kBig = Buf::kBig;
    const WalkParams<T>& P;
    WsPair<KIND, T, CONS>& W;
    WalkBuf<KIND, T>* B = nullptr;
    WalkRanges* Rg;
    v2_t<T> H;
    vec4_t<T> box;
    int nf = 0, nn = 0, nb = 0;
    int g = 0;
    uint32_t use = 0;  // slots handed over so far
    bool alive = true;
    uint32_t* rec = nullptr;  // the group's kept interaction list, or null
    int rec_n = 0, rec_cap = 0;

    LENS_DEV WsProducer(const WalkParams<T>& p, WsPair<KIND, T, CONS>& w) : P(p), W(w), Rg(&w.rng) {}

    // Take the next slot, waiting until the consumer has released it.
    LENS_DEV void acquire()
    {
        const int s = use & 1;
        if (use >= 2 && alive) alive = mbar_wait(&W.empty[s], ((use >> 1) - 1) & 1, P.err, P.wait_cycles);
        B = &W.slot[s].buf;
        nf = nn = nb = 0;
    }
    // Publish the current slot with its counts.
    LENS_DEV void handoff(int flags)
    {
        const int s = use & 1;
        if (!alive) {
            // the consumer is gone: keep writing into this slot, publish nothing
            nf = nn = nb = 0;
            return;
        }
        __syncwarp();
        if ((threadIdx.x & 31) == 0) {
            WsSlot<KIND, T>& sl = W.slot[s];
            sl.nf = nf;
            sl.nn = nn;
            sl.nb = nb;
            sl.g = g;
            sl.flags = flags;
        }
        mbar_arrive(&W.full[s]);
        ++use;
    }
    LENS_DEV void flush()
    {
        handoff(0);
        acquire();
    }
    LENS_DEV void flush_far() { flush(); }
    LENS_DEV void flush_near() { flush(); }
    LENS_DEV void flush_big() { flush(); }
};

template <int KIND, typename T, int CONS>
LENS_DEV void ws_produce(const WalkParams<T>& P, WsPair<KIND, T, CONS>& W, int* stack)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    WsProducer<KIND, T, CONS> C(P, W);
    for (;;) {
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(P.counter, 1u);
        g = __shfl_sync(full, g, 0);
        C.acquire();
        if (!C.alive) return;
        if ((int64_t)g >= P.n_groups) {
            C.handoff(kWsStop);
            return;
        }
        if (P.order) g = P.order[g];
        C.g = (int)g;
        C.H = P.gH[g];
        C.box = P.gbox[g];
        int c_vis = 0, c_acc = 0, c_near = 0, c_bigs = 0, c_bigk = 0;
        C.rec = P.list_ids ? P.list_ids + (int64_t)g * P.list_K : nullptr;
        C.rec_n = 0;
        C.rec_cap = P.list_K;
        const bool whole = traverse(C, stack, c_vis, c_acc, c_near, c_bigs, c_bigk);
        C.handoff(kWsLast);
        if (!C.alive) return;
        if (C.rec && lane == 0) P.list_n[g] = whole && C.rec_n <= C.rec_cap ? (uint32_t)C.rec_n : kListOverflow;
        if (P.gcost && lane == 0) P.gcost[g] += (uint32_t)(c_vis + c_acc + c_near + c_bigk);
        if (P.stats && lane == 0) {
            unsigned long long nr = P.grange[g].y;
            atomicAdd(&P.stats[0], 1ull);
            atomicAdd(&P.stats[1], (unsigned long long)c_vis);
            atomicAdd(&P.stats[2], (unsigned long long)c_acc);
            atomicAdd(&P.stats[3], (unsigned long long)c_near);
            atomicAdd(&P.stats[4], (unsigned long long)c_bigs);
            atomicAdd(&P.stats[5], (unsigned long long)c_bigk);
            atomicAdd(&P.stats[6], nr * (unsigned long long)(c_acc + c_near + c_bigk));
        }
    }
}

// Consumer rank c of its team: rays c * 32 + [0, 32 R) of every group.
template <int KIND, typename T, int R, bool AO, int CONS>
LENS_DEV void ws_consume(const WalkParams<T>& P, WsPair<KIND, T, CONS>& W, int c)
{
    const int lane = threadIdx.x & 31;
    WalkEval<KIND, T, R, AO> E(P, &W.slot[0].buf, &W.tot[c]);
    uint32_t ridx[R];
    bool rv[R];
    int cur = -1;
    uint2 rg = make_uint2(0, 0);
    for (uint32_t use = 0;; ++use) {
        const int s = use & 1;
        if (!mbar_wait(&W.full[s], (use >> 1) & 1, P.err, P.wait_cycles)) return;
        const WsSlot<KIND, T>& sl = W.slot[s];
        const int flags = sl.flags, g = sl.g;
        if (flags & kWsStop) return;
        if (g != cur) {
            // the group's first slot: load its rays
            cur = g;
            E.H = P.gH[g];
            E.box = P.gbox[g];
            rg = P.grange[g];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                int k = c * 32 + r * 32 + lane;
                rv[r] = k < (int)rg.y;
                if (rv[r]) {
                    v2_t<T> l = P.ray_l[rg.x + k];
                    E.lx[r] = l.x;
                    E.ly[r] = l.y;
                    ridx[r] = P.ray_idx[rg.x + k];
                } else {
                    E.lx[r] = E.box.x;
                    E.ly[r] = E.box.y;
                    ridx[r] = 0;
                }
                E.part[r].zero();
            }
            E.tot_zero();
        }
        E.B = &W.slot[s].buf;
        const int nf = sl.nf, nn = sl.nn, nb = sl.nb;
        if (nf) E.eval_far(nf);
        if (nn) E.eval_near(nn);
        if constexpr (KIND != LENS_POINT)
            if (nb) E.eval_big(nb);
        __syncwarp();
        mbar_arrive(&W.empty[s]);
        if (flags & kWsLast) {
            if (P.n_halos > 0) E.halos();
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (!rv[r]) continue;
                uint32_t i = ridx[r];
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    if (AO && q >= 2) break;
                    T val = E.tot_get(r, q);
                    if (P.accumulate) val += P.out[q][i];
                    P.out[q][i] = val;
                }
            }
            cur = -1;
            __syncwarp();
        }
    }
}

template <int KIND, typename T, int R, bool AO, int CONS>
__global__ void __launch_bounds__(WsShape<CONS>::kThreads, WsShape<CONS>::kBlocksPerSm)
walk_ws_kernel(WalkParams<T> P)
{
    using Sh = WsShape<CONS>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int team = warp % kWsPairs, role = warp / kWsPairs;  // role 0: producer; 1..CONS: consumers
    WsPair<KIND, T, CONS>& W = reinterpret_cast<WsPair<KIND, T, CONS>*>(smem_raw)[team];
    if (role == 0 && lane == 0) {
        mbar_init(&W.full[0], 32);
        mbar_init(&W.full[1], 32);
        mbar_init(&W.empty[0], 32 * CONS);
        mbar_init(&W.empty[1], 32 * CONS);
    }
    __syncthreads();
    if (role == 0) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(Sh::kProdRegs));
        int* stack = P.stack + ((int64_t)blockIdx.x * kWsPairs + team) * kStackCap;
        ws_produce<KIND, T, CONS>(P, W, stack);
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(Sh::kConsRegs));
        ws_consume<KIND, T, R, AO, CONS>(P, W, role - 1);
    }
}

template <int KIND, typename T, int R, bool AO, int CONS>
static int ws_blocks_per_sm()
{
    static int cached = -1;
    if (cached < 0) {
        size_t smem = kWsPairs * sizeof(WsPair<KIND, T, CONS>);
        cudaFuncSetAttribute(walk_ws_kernel<KIND, T, R, AO, CONS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        cudaFuncSetAttribute(walk_ws_kernel<KIND, T, R, AO, CONS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             100);
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, walk_ws_kernel<KIND, T, R, AO, CONS>,
                                                      WsShape<CONS>::kThreads, smem);
        cached = nb > 0 ? nb : 1;
    }
    return cached;
}

// Compiled registers per thread of the kernel (the register split is only
// valid if the launch holds exactly kLaunchRegs per thread).
template <int KIND, typename T, int R, bool AO, int CONS>
static int ws_kernel_regs()
{
    static int cached = -1;
    if (cached < 0) {
        cudaFuncAttributes a{};
        cached = cudaFuncGetAttributes(&a, walk_ws_kernel<KIND, T, R, AO, CONS>) == cudaSuccess ? a.numRegs : 0;
    }
    return cached;
}

template <int KIND, typename T, int R, bool AO, int CONS>
static bool ws_launch_one(const WalkParams<T>& P, int num_sms, cudaStream_t s)
{
    if (ws_kernel_regs<KIND, T, R, AO, CONS>() != WsShape<CONS>::kLaunchRegs) return false;
    size_t smem = kWsPairs * sizeof(WsPair<KIND, T, CONS>);
    int bps = ws_blocks_per_sm<KIND, T, R, AO, CONS>();
    // stacks are allocated for 16 blocks x kWalkWarps warps per SM
    if (bps > 16 * kWalkWarps / kWsPairs) bps = 16 * kWalkWarps / kWsPairs;
    { walk_ws_kernel<KIND, T, R, AO, CONS><<<num_sms * bps, WsShape<CONS>::kThreads, smem, s>>>(P); note_launch(); }
    return true;
}

template <typename T, int R, int CONS>
static bool launch_kind_ws(int kind, bool ao, const WalkParams<T>& P, int num_sms, cudaStream_t s)
{
    if (kind == LENS_POINT)
        return ao ? ws_launch_one<LENS_POINT, T, R, true, CONS>(P, num_sms, s)
                  : ws_launch_one<LENS_POINT, T, R, false, CONS>(P, num_sms, s);
    if (kind == LENS_GAUSS)
        return ao ? ws_launch_one<LENS_GAUSS, T, R, true, CONS>(P, num_sms, s)
                  : ws_launch_one<LENS_GAUSS, T, R, false, CONS>(P, num_sms, s);
    return ao ? ws_launch_one<LENS_NFW, T, R, true, CONS>(P, num_sms, s)
              : ws_launch_one<LENS_NFW, T, R, false, CONS>(P, num_sms, s);
}

// R: rays per lane of the group (32 R rays).  consumers = 2 splits a 64-ray
// group between two consumer warps (R = 2 only).
template <typename T, int R>
bool launch_ws(int kind, bool ao, const WalkParams<T>& P, int num_sms, cudaStream_t s, int consumers)
{
    if constexpr (R == 2) {
        if (consumers == 2) return launch_kind_ws<T, 1, 2>(kind, ao, P, num_sms, s);
    }
    return launch_kind_ws<T, R, 1>(kind, ao, P, num_sms, s);
}

template bool launch_ws<float, 1>(int, bool, const WalkParams<float>&, int, cudaStream_t, int);
template bool launch_ws<float, 2>(int, bool, const WalkParams<float>&, int, cudaStream_t, int);
template bool launch_ws<double, 1>(int, bool, const WalkParams<double>&, int, cudaStream_t, int);
template bool launch_ws<double, 2>(int, bool, const WalkParams<double>&, int, cudaStream_t, int);

}  // namespace lens
