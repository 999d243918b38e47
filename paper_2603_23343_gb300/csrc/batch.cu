// Many independent Jacobi-PCG problems (Sec. VII's solver, one per grid) in
// ONE persistent kernel launch.
//
// The grid is as many CTAs as the GPU holds at once (a cooperative launch,
// so every CTA is resident).  Setup and finalize are phases of all problems
// at once, separated by grid-wide barriers:
//
//   reset states | max |b| | r0 = b - A x0 (FP64) | phase control    once
//   ... every problem through its own phases, no barrier ...
//   x += d + alpha p | true residual (FP64)                           once
//
// In between, each problem runs its own sequence of phases: pass A, pass B,
// pass A, ... and, when a pass B asks for a residual replacement, a flush
// and an FP64 residual before the next pass A.  A phase is a set of work
// items: a pass item is one (x, y) tile of the problem marched through a
// run of z planes (the same z-marching code as the single-problem passes,
// engine.cuh), a row item a run of grid rows.  Any CTA claims any available
// item of any unfinished problem (an atomic counter in the problem's claim
// word, whose upper half holds the phase's item count), preferring the problem it
// worked on last; the CTA that completes a phase's last item adds the
// problem's partial sums in item order (bitwise reproducible), takes the
// scalar step (alpha; beta, convergence, the replacement trigger) and opens
// the problem's next phase.  So one problem's pass B runs while another's
// pass A does, a finished problem drops out, and no CTA waits for work
// while any is available.  The z depth of a pass item is chosen when its
// phase opens: about two items per CTA over the unfinished problems, 4 to 32
// planes.
//
// Every wait is bounded: the grid barrier (a counter and a generation word)
// after kBarrierPolls polls, a CTA finding no work after kIdlePolls tries;
// either raises an abort flag that every CTA checks, and the problems that
// had not finished report GBPCG_TIMEOUT.
#include <algorithm>
#include <cstring>
#include <list>
#include <mutex>
#include <vector>

#include "solver.cuh"

namespace gb {

namespace {

// The solver scalars are shared between SMs within this launch: they are
// read and written through volatile accesses (never a stale L1 line).
__device__ __forceinline__ volatile SolveState *vol(SolveState *s) { return s; }

constexpr int kBatchThreads = 256;
constexpr int kBatchZDepth = 32;  // most z planes per pass item
constexpr int kRowPoints = 16384;  // grid points per row item (at least one row)
constexpr uint32_t kBarrierPolls = 1u << 22;  // x ~64 ns of sleep: well under a second
constexpr int kBatchMaxProblems = 4096;
constexpr uint32_t kIdlePolls = 1u << 21;  // claims that found no work in a row (~0.5 us each): about a second

// Tile configurations of the persistent kernel (all 256 threads: the FP64
// residual code strides rows by 256 threads).
enum BatchCfg { BC_64x16 = 0, BC_128x8 = 1, BC_32x32 = 2, BC_COUNT = 3 };
struct BcDims { int tx, ty; };
inline BcDims bc_dims(int c) { return c == BC_64x16 ? BcDims{64, 16} : c == BC_128x8 ? BcDims{128, 8} : BcDims{32, 32}; }

struct __align__(128) BatchProblem {
    CUtensorMap hz, hp0, hp1;  // halo boxes of z, p0, p1
    CUtensorMap cd, cz;        // centre boxes of d (pass A) and z (pass B)
    OpConst op;
    int nx, ny, nz, tiles_x, tiles;
    int row0_item, nrow_items;  // row items
    int rows_per_item;
    float *z, *p0, *p1, *d;
    SolveState *st;
    double *partials;
    Res64Args ra;
};

struct __align__(64) BatchHeader {
    unsigned bar_count;
    unsigned bar_gen;
    int abort;
    int phases;              // phases run over all problems
    int active;              // problems not yet finished
    int pad;
    long long tile_planes;   // sum over unfinished problems of tiles x planes
};

// What a problem's current phase is (its work items are claimed through
// ProbCtl::claim).
enum PhaseKind { PH_A = 0, PH_B = 1, PH_FLUSH = 2, PH_RESID = 3, PH_DONE = 4 };

struct __align__(64) ProbCtl {
    // (items of the current phase << 32) | items of it claimed so far: one atomic add returns
    // an index together with the item count of the phase it belongs to, so a claim that
    // overshoots a phase can never be mistaken for an item of the phase opened after it
    unsigned long long claim;
    int kind;                  // PhaseKind of the current phase
    int nitems;                // its work items
    int depth;                 // pass phases: z planes per item
    int phases;                // phases this problem has run
};

struct BatchArgs {
    BatchProblem *probs;
    ProbCtl *ctl;
    const int *row_prob;   // row item -> problem
    BatchHeader *hdr;
    int nprob, nrow_items;
    double tol;
    int maxit;
    int depth0;            // z planes per item of the first pass phase
};

// Grid-wide barrier (bounded): false once any CTA has given up.
__device__ __forceinline__ bool batch_barrier(BatchHeader *h) {
    // writes of this phase (generic proxy) before the next phase's TMA loads (async proxy)
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __threadfence();
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &h->bar_gen;
        volatile int *abort = &h->abort;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(&h->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&h->bar_count, 0u);
            __threadfence();
            atomicAdd(&h->bar_gen, 1u);
        } else {
            uint32_t polls = 0;
            while (*gen == g) {
                if (*abort) break;
                if (++polls > kBarrierPolls) {
                    atomicExch(&h->abort, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");
        s_ok = *abort == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// The whole batch.  X: type of b and x (float or double).
template <int TX, int TY, int S, typename X>
__global__ void __launch_bounds__(kBatchThreads, 3) batch_kernel(const BatchArgs A) {
    using T = float;
    using GA = Geometry<T, TX, TY, K_PASSA>;
    using GB = Geometry<T, TX, TY, K_PASSB>;
    static_assert(GA::NT == kBatchThreads, "persistent tiles have 256 threads");
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[S];
    __shared__ int s_timeout;
    BatchHeader *hdr = A.hdr;
    if (threadIdx.x == 0) {
        s_timeout = 0;
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t ring = 0;  // loads this CTA has issued into its ring (stage and phase of the next one)
    const unsigned G = gridDim.x;

    // ---- reset every problem's state ----
    for (int p = blockIdx.x; p < A.nprob; p += G)
        if (threadIdx.x == 0) {
            SolveState *st = A.probs[p].st;
            memset(st, 0, sizeof(SolveState));
            st->tol2 = A.tol * A.tol;
            st->maxit = A.maxit;
            st->status = GBPCG_NOT_CONVERGED;
        }
    if (!batch_barrier(hdr)) return;

    // ---- max |b| per problem (bit patterns: integer maxima) ----
    for (int item = blockIdx.x; item < A.nrow_items; item += G) {
        const BatchProblem &P = A.probs[A.row_prob[item]];
        const int local = item - P.row0_item;
        const int r0 = local * P.rows_per_item, r1 = min(P.ny * P.nz, r0 + P.rows_per_item);
        using U = typename std::conditional<sizeof(X) == 8, unsigned long long, unsigned int>::type;
        constexpr U kAbs = (U)~((U)1 << (8 * sizeof(X) - 1));
        const X *b = static_cast<const X *>(P.ra.b);
        U m = 0;
        for (int row = r0; row < r1; ++row)
            for (int i = threadIdx.x; i < P.nx; i += kBatchThreads) {
                X v = __ldg(b + (int64_t)row * P.nx + i);
                U u;
                memcpy(&u, &v, sizeof(U));
                u &= kAbs;
                m = u > m ? u : m;
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const U t = __shfl_xor_sync(0xffffffffu, m, o);
            m = t > m ? t : m;
        }
        if ((threadIdx.x & 31) == 0 && m) {
            X v;
            memcpy(&v, &m, sizeof(U));
            atomicMax(&P.st->rhs_bits, (unsigned long long)__double_as_longlong((double)v));
        }
    }
    if (!batch_barrier(hdr)) return;

    // ---- r0 = b - A x0 in FP64, z0 = D^-1 r0, d = 0 ----
    for (int item = blockIdx.x; item < A.nrow_items; item += G) {
        const BatchProblem &P = A.probs[A.row_prob[item]];
        const int local = item - P.row0_item;
        const int r0 = local * P.rows_per_item, r1 = min(P.ny * P.nz, r0 + P.rows_per_item);
        double part[3], tot[3], unscale;
        res64_rows<RES_INIT, X, X, false, T, true>(P.ra, r0, r1, 1, part, &unscale);
        if (group_sum_last<3, kBatchThreads>(part, P.partials, &P.st->ticket[4 + RES_INIT], local, P.nrow_items,
                                             tot) &&
            threadIdx.x == 0)
            res64_finish<RES_INIT>(vol(P.st), tot, unscale);
    }
    if (!batch_barrier(hdr)) return;

    // ---- the iterations: every problem advances through its own phases ----
    // pass A -> pass B -> pass A ..., or after a pass B that asked for a residual replacement,
    // flush -> FP64 residual -> pass A.  A phase is a set of work items (tiles of z planes, or
    // runs of rows); any CTA claims any available item of any problem, and the CTA that
    // completes a phase's last item takes the problem's scalar step and opens its next phase.
    // No barrier separates problems: one problem's pass B runs while another's pass A does.
    for (int p = blockIdx.x; p < A.nprob; p += G)
        if (threadIdx.x == 0) {
            const BatchProblem &P = A.probs[p];
            ProbCtl &c = A.ctl[p];
            const bool fin = vol(P.st)->done != 0;
            const int need = (2 * P.tiles * P.nz + 4 * (int)kMaxPassBlocks - 1) / (4 * (int)kMaxPassBlocks);
            const int dep = min(P.nz, max(A.depth0, need));
            c.kind = fin ? PH_DONE : PH_A;
            c.depth = dep;
            c.nitems = fin ? 0 : P.tiles * ((P.nz + dep - 1) / dep);
            c.phases = 0;
            c.claim = (unsigned long long)(unsigned)c.nitems << 32;
            if (!fin) {
                atomicAdd(&hdr->active, 1);
                atomicAdd((unsigned long long *)&hdr->tile_planes, (unsigned long long)((long long)P.tiles * P.nz));
            }
        }
    if (!batch_barrier(hdr)) return;

    // z planes per pass item of a phase opening now: about two items per CTA over the
    // unfinished problems' tile-planes, 4 to 32 planes, and enough planes that the problem's
    // pass-B partial sums fit its slots
    auto pass_depth = [&](const BatchProblem &P) {
        const long long tp = ((volatile long long *)&hdr->tile_planes)[0];
        const int d = (int)max(4LL, min((long long)kBatchZDepth, (tp + 2LL * G - 1) / (2LL * G)));
        const int need = (2 * P.tiles * P.nz + 4 * (int)kMaxPassBlocks - 1) / (4 * (int)kMaxPassBlocks);
        return min(P.nz, max(d, need));
    };
    // thread 0 of the CTA that completed a phase: open the problem's next phase
    auto advance = [&](ProbCtl *c, const BatchProblem &P, int next) {
        int n = 0, d = c->depth;
        if (next == PH_A) {
            d = pass_depth(P);
            n = P.tiles * ((P.nz + d - 1) / d);
        } else if (next == PH_B) {
            n = P.tiles * ((P.nz + d - 1) / d);
        } else if (next == PH_FLUSH || next == PH_RESID) {
            n = P.nrow_items;
        } else {
            atomicSub(&hdr->active, 1);
            atomicAdd((unsigned long long *)&hdr->tile_planes, (unsigned long long)(-(long long)P.tiles * P.nz));
        }
        c->kind = next;
        c->nitems = n;
        c->depth = d;
        c->phases += 1;
        atomicAdd(&hdr->phases, 1);
        __threadfence();
        atomicExch(&c->claim, (unsigned long long)(unsigned)n << 32);
    };

    __shared__ int s_p, s_i, s_q;
    int cur = (int)(blockIdx.x % (unsigned)A.nprob);
    uint32_t idle = 0;
    for (;;) {
        // claim a work item: warp 0 looks at every problem from the last one this CTA worked on
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int got_p = -1, got_i = 0;
            for (int base = 0; base < A.nprob && got_p < 0; base += 32) {
                const int q = base + lane;
                bool cand = false;
                if (q < A.nprob) {
                    int p = cur + q;
                    if (p >= A.nprob) p -= A.nprob;
                    const unsigned long long w = ((volatile unsigned long long *)&A.ctl[p].claim)[0];
                    cand = (unsigned)w < (unsigned)(w >> 32);
                }
                unsigned m = __ballot_sync(0xffffffffu, cand);
                if (lane == 0) {
                    while (m && got_p < 0) {
                        const int bit = __ffs(m) - 1;
                        m &= m - 1;
                        int p = cur + base + bit;
                        if (p >= A.nprob) p -= A.nprob;
                        ProbCtl *c = &A.ctl[p];
                        const unsigned long long old = atomicAdd(&c->claim, 1ull);
                        __threadfence();
                        // an index below the count in the same word is an item of the phase
                        // that word belongs to; that phase cannot close before the item
                        // completes, so the kind and depth read afterwards are its own
                        if ((unsigned)old < (unsigned)(old >> 32)) {
                            got_p = p;
                            got_i = (int)(unsigned)old;
                        }
                    }
                }
                got_p = __shfl_sync(0xffffffffu, got_p, 0);
                got_i = __shfl_sync(0xffffffffu, got_i, 0);
            }
            if (lane == 0) {
                s_p = got_p;
                s_i = got_i;
                // with nothing claimed, thread 0 alone reads whether the batch has finished or
                // given up: warps that read `active` at different moments would leave the loop at
                // different __syncthreads, and the CTA's warps would then run out of step with
                // one another across the grid barriers that follow
                s_q = got_p >= 0 ? 0
                      : ((volatile int *)&hdr->active)[0] == 0 ? 1
                      : ((volatile int *)&hdr->abort)[0] ? 2 : 0;
            }
        }
        __syncthreads();
        const int pi = s_p, local = s_i, quit = s_q;
        __syncthreads();  // s_p, s_i and s_q are written again at the next claim
        if (pi < 0) {
            if (quit == 1) break;
            if (quit == 2) return;
            if (++idle > kIdlePolls) {
                if (threadIdx.x == 0) atomicExch(&hdr->abort, 1);
                return;
            }
            __nanosleep(256);
            continue;
        }
        idle = 0;
        cur = pi;
        // stores of the phase before (other CTAs, generic proxy) before this item's TMA loads
        asm volatile("fence.proxy.async.global;" ::: "memory");
        const BatchProblem &P = A.probs[pi];
        SolveState *st = P.st;
        ProbCtl *ctl = &A.ctl[pi];
        const int kind = ((volatile int *)&ctl->kind)[0];
        const int nit = ((volatile int *)&ctl->nitems)[0];
        const int dep = ((volatile int *)&ctl->depth)[0];
        if (kind == PH_A || kind == PH_B) {
            const int tile = local % P.tiles, chunk = local / P.tiles;
            const int x0 = (tile % P.tiles_x) * TX, y0 = (tile / P.tiles_x) * TY;
            const int k0 = chunk * dep, k1 = min(P.nz, k0 + dep);
            if (kind == PH_A) {
                // p_k = z_k + beta p_{k-1}, d += alpha_{k-1} p_{k-1}, p.Ap
                const MarchScalars sc = read_scalars<K_PASSA>(vol(st));
                const bool odd = sc.it & 1;
                MarchIO<T, K_PASSA> io;
                io.H0 = P.z;
                io.H1 = odd ? P.p0 : P.p1;  // p_{k-1}
                io.C0 = P.d;
                io.O0 = odd ? P.p1 : P.p0;  // p_k
                io.O1 = P.d;
                io.M0 = &P.hz;
                io.M1 = odd ? &P.hp0 : &P.hp1;
                io.MC = &P.cd;
                float acc[GA::NV];
                acc[0] = 0.f;
                ring += march_tile<T, TX, TY, S, K_PASSA, true, OpConst, false>(smem, full, &s_timeout, ring, io,
                                                                               P.op, P.nx, P.ny, P.nz, x0, y0, k0,
                                                                               k1, sc, acc);
                if (s_timeout) {
                    if (threadIdx.x == 0) atomicExch(&hdr->abort, 1);
                    return;
                }
                asm volatile("fence.proxy.async.global;" ::: "memory");
                double part[1], tot[1];
                block_sum<1, kBatchThreads>(acc, part);
                if (group_sum_last<1, kBatchThreads>(part, P.partials, &st->ticket[K_PASSA], local, nit, tot) &&
                    threadIdx.x == 0) {
                    passa_finish(vol(st), tot[0], false);
                    advance(ctl, P, vol(st)->done ? PH_DONE : PH_B);
                }
            } else {
                // q = A p_k, r = D z - alpha q, z = D^-1 r, r.r, r.z
                const MarchScalars sc = read_scalars<K_PASSB>(vol(st));
                const bool odd = sc.it & 1;
                MarchIO<T, K_PASSB> io;
                io.H0 = odd ? P.p1 : P.p0;  // p_k
                io.H1 = io.H0;
                io.C0 = P.z;
                io.O0 = P.z;
                io.O1 = P.z;
                io.M0 = odd ? &P.hp1 : &P.hp0;
                io.M1 = io.M0;
                io.MC = &P.cz;
                float acc[GB::NV];
                acc[0] = acc[1] = 0.f;
                ring += march_tile<T, TX, TY, S, K_PASSB, true, OpConst, false>(smem, full, &s_timeout, ring, io,
                                                                               P.op, P.nx, P.ny, P.nz, x0, y0, k0,
                                                                               k1, sc, acc);
                if (s_timeout) {
                    if (threadIdx.x == 0) atomicExch(&hdr->abort, 1);
                    return;
                }
                asm volatile("fence.proxy.async.global;" ::: "memory");
                double part[2], tot[2];
                block_sum<2, kBatchThreads>(acc, part);
                if (group_sum_last<2, kBatchThreads>(part, P.partials, &st->ticket[K_PASSB], local, nit, tot) &&
                    threadIdx.x == 0) {
                    passb_finish(vol(st), sc.it, tot[0], tot[1], false);
                    advance(ctl, P, vol(st)->done ? PH_DONE : vol(st)->replace ? PH_FLUSH : PH_A);
                }
            }
        } else {
            const int r0 = local * P.rows_per_item, r1 = min(P.ny * P.nz, r0 + P.rows_per_item);
            if (kind == PH_FLUSH) {
                // x += (d + alpha_{k-1} p_{k-1}) / s, d = 0
                const volatile SolveState *vs = vol(st);
                const T *p = ((vs->it - 1) & 1) ? P.p1 : P.p0;
                const float a = vs->pending ? (float)vs->alpha : 0.0f;
                const double inv_s = 1.0 / rhs_scale(vs->rhs_bits);
                X *x = static_cast<X *>(const_cast<void *>(P.ra.x));
                const X is = (X)inv_s;
                // p, d and x were written in this launch by other SMs: loads through L2 only
                for (int64_t g = (int64_t)r0 * P.nx + threadIdx.x; g < (int64_t)r1 * P.nx; g += kBatchThreads) {
                    const X inc = (X)fmaf(a, __ldcg(p + g), __ldcg(P.d + g));
                    const X xo = __ldcg(x + g);
                    x[g] = inv_s == 1.0 ? xo + inc : xo + inc * is;
                    P.d[g] = 0.0f;
                }
                // the next pass A reads d through the TMA (async proxy)
                asm volatile("fence.proxy.async.global;" ::: "memory");
                __threadfence();
                __syncthreads();
                const double part[1] = {0.0};
                double tot[1];
                if (group_sum_last<1, kBatchThreads>(part, P.partials, &st->ticket[0], local, nit, tot) &&
                    threadIdx.x == 0)
                    advance(ctl, P, PH_RESID);
            } else {
                // r = b - A x in FP64, z = D^-1 r, the replacement's decisions
                double part[2], tot[2], unscale;
                res64_rows<RES_REPLACE, X, X, false, T, true>(P.ra, r0, r1, 1, part, &unscale);
                asm volatile("fence.proxy.async.global;" ::: "memory");  // z, read by the next pass A's TMA
                if (group_sum_last<2, kBatchThreads>(part, P.partials, &st->ticket[4 + RES_REPLACE], local, nit,
                                                     tot) &&
                    threadIdx.x == 0) {
                    res64_finish<RES_REPLACE>(vol(st), tot, unscale);
                    advance(ctl, P, vol(st)->done ? PH_DONE : PH_A);
                }
            }
        }
    }
    if (!batch_barrier(hdr)) return;

    // ---- x += (d + alpha_{k-1} p_{k-1}) / s (x = 0 when b = 0) ----
    for (int item = blockIdx.x; item < A.nrow_items; item += G) {
        const BatchProblem &P = A.probs[A.row_prob[item]];
        const volatile SolveState *st = vol(P.st);
        const int local = item - P.row0_item;
        const int r0 = local * P.rows_per_item, r1 = min(P.ny * P.nz, r0 + P.rows_per_item);
        X *x = static_cast<X *>(const_cast<void *>(P.ra.x));
        if (st->zero_x) {
            for (int64_t g = (int64_t)r0 * P.nx + threadIdx.x; g < (int64_t)r1 * P.nx; g += kBatchThreads) x[g] = X(0);
            continue;
        }
        const T *p = ((st->it - 1) & 1) ? P.p1 : P.p0;
        const float a = st->pending ? (float)st->alpha : 0.0f;
        const double inv_s = 1.0 / rhs_scale(st->rhs_bits);
        const X is = (X)inv_s;
        // p, d and x were written in this launch by other SMs: loads through L2 only
        for (int64_t g = (int64_t)r0 * P.nx + threadIdx.x; g < (int64_t)r1 * P.nx; g += kBatchThreads) {
            const X inc = (X)fmaf(a, __ldcg(p + g), __ldcg(P.d + g));
            const X xo = __ldcg(x + g);
            x[g] = inv_s == 1.0 ? xo + inc : xo + inc * is;
        }
    }
    if (!batch_barrier(hdr)) return;

    // ---- true residual ||b - A x|| in FP64 (unless a replacement already evaluated this x) ----
    for (int item = blockIdx.x; item < A.nrow_items; item += G) {
        const BatchProblem &P = A.probs[A.row_prob[item]];
        SolveState *st = P.st;
        if (vol(st)->true_known) continue;
        const int local = item - P.row0_item;
        const int r0 = local * P.rows_per_item, r1 = min(P.ny * P.nz, r0 + P.rows_per_item);
        double part[1], tot[1], unscale;
        res64_rows<RES_TRUE, X, X, false, T, true>(P.ra, r0, r1, 1, part, &unscale);
        if (group_sum_last<1, kBatchThreads>(part, P.partials, &st->ticket[4 + RES_TRUE], local, P.nrow_items, tot) &&
            threadIdx.x == 0)
            res64_finish<RES_TRUE>(vol(st), tot, unscale);
    }
}

// Kernel, shared memory and occupancy of one configuration and io type.
struct BatchKernel {
    void *fn = nullptr;
    size_t smem = 0;
};

template <int TX, int TY, typename X>
BatchKernel batch_kernel_of() {
    constexpr int S = 4;
    BatchKernel k;
    k.fn = reinterpret_cast<void *>(&batch_kernel<TX, TY, S, X>);
    k.smem = zmarch_smem_bytes<float, TX, TY, S, K_PASSA>();
    return k;
}

template <typename X>
BatchKernel batch_kernel_for(int cfg) {
    switch (cfg) {
        case BC_64x16: return batch_kernel_of<64, 16, X>();
        case BC_128x8: return batch_kernel_of<128, 8, X>();
        default: return batch_kernel_of<32, 32, X>();
    }
}

// Geometry of one problem under a configuration (pass items: a pass phase
// chooses its z depth when it opens; row items: set-up, flush, FP64 residual
// and finalize).
struct ProbGeom {
    int tiles_x, tiles, rows_per_item, nrow_items;
};
ProbGeom prob_geom(const gbpcg_grid &g, int cfg) {
    const BcDims d = bc_dims(cfg);
    ProbGeom p;
    p.tiles_x = (g.nx + d.tx - 1) / d.tx;
    p.tiles = p.tiles_x * ((g.ny + d.ty - 1) / d.ty);
    // at least kRowPoints points per row item, and few enough items for the partial-sum slots
    p.rows_per_item = std::max({1, kRowPoints / g.nx, (g.ny * g.nz + 4095) / 4096});
    p.nrow_items = (g.ny * g.nz + p.rows_per_item - 1) / p.rows_per_item;
    return p;
}

struct BatchLayout {
    size_t hdr, probs, ctl, rows, total;
};

// The batch's own region at the front of the workspace: header, problem
// table, per-problem phase control and the row-item-to-problem map.
BatchLayout batch_layout(int nprob, const gbpcg_grid *grids) {
    BatchLayout L;
    int rows = 0;
    for (int i = 0; i < nprob; ++i) rows += prob_geom(grids[i], 0).nrow_items;  // the same for every cfg
    size_t o = 0;
    L.hdr = o; o += round256(sizeof(BatchHeader));
    L.probs = o; o += round256(sizeof(BatchProblem) * (size_t)nprob);
    L.ctl = o; o += round256(sizeof(ProbCtl) * (size_t)nprob);
    L.rows = o; o += round256(sizeof(int) * (size_t)rows);
    L.total = o;
    return L;
}

// Instantiated single-kernel graphs, keyed by everything they bake in.
struct PersistKey {
    std::vector<SolveKey> keys;
    int cfg;
};
struct PersistGraph {
    PersistKey key;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};
std::mutex g_persist_mu;
std::list<PersistGraph> g_persist;
constexpr size_t kPersistMax = 8;

bool same_key(const PersistKey &a, const PersistKey &b) {
    if (a.cfg != b.cfg || a.keys.size() != b.keys.size()) return false;
    for (size_t i = 0; i < a.keys.size(); ++i)
        if (!(a.keys[i] == b.keys[i])) return false;
    return true;
}

}  // namespace

bool batch_persistent_ok(int nprob, const gbpcg_grid *grids) {
    if (nprob > kBatchMaxProblems) return false;
    for (int i = 0; i < nprob; ++i) {
        const gbpcg_grid &g = grids[i];
        if (g.k_block || g.nx % 4) return false;  // Poisson operator, 16-byte rows for the TMA boxes
        for (int c = 0; c < BC_COUNT; ++c)  // the pass depth keeps every item count within the partial-sum slots
            if (prob_geom(g, c).tiles > 4096) return false;
    }
    return true;
}

size_t batch_persistent_bytes(int nprob, const gbpcg_grid *grids) { return batch_layout(nprob, grids).total; }

int batch_persistent_cfgs() { return BC_COUNT; }

// Sets up the problem table in the workspace's batch region and launches the
// persistent kernel (inside a cached one-node CUDA graph when the cooperative
// launch can be captured, else directly).  calls[i] describes problem i
// (its workspace piece, b, x); maxit caps each problem's iterations.
int batch_persistent_launch(int nprob, const gbpcg_grid *grids, const SolveCall *calls, char *region, int cfg,
                            double tol, int maxit, int io, cudaStream_t s) {
    const BatchLayout BL = batch_layout(nprob, grids);
    const BcDims dims = bc_dims(cfg);
    std::vector<BatchProblem> probs(nprob);
    std::vector<int> row_prob;
    int nrow = 0;
    for (int i = 0; i < nprob; ++i) {
        const gbpcg_grid &g = grids[i];
        const SolveCall &c = calls[i];
        const ProbGeom pg = prob_geom(g, cfg);
        BatchProblem &P = probs[i];
        memset(&P, 0, sizeof(P));
        char *w = c.ws;
        P.z = reinterpret_cast<float *>(w + c.L.z);
        P.p0 = reinterpret_cast<float *>(w + c.L.p0);
        P.p1 = reinterpret_cast<float *>(w + c.L.p1);
        P.d = reinterpret_cast<float *>(w + c.L.d);
        P.st = reinterpret_cast<SolveState *>(w + c.L.state);
        P.partials = reinterpret_cast<double *>(w + c.L.partials);
        if (!tma_ok(sizeof(float), g.nx, {P.z, P.p0, P.p1, P.d}))
            return fail_arg("persistent batch: every grid needs nx a multiple of 4 (16-byte rows)");
        // halo boxes (TX + 2 XH) x (TY + 2), centre boxes TX x TY, as the single-problem passes use
        const int xh = 4;
        int rc = 0;
        rc |= make_map_3d(&P.hz, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, P.z, g.nx, g.ny, g.nz, dims.tx + 2 * xh,
                          dims.ty + 2, 1);
        rc |= make_map_3d(&P.hp0, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, P.p0, g.nx, g.ny, g.nz, dims.tx + 2 * xh,
                          dims.ty + 2, 1);
        rc |= make_map_3d(&P.hp1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, P.p1, g.nx, g.ny, g.nz, dims.tx + 2 * xh,
                          dims.ty + 2, 1);
        rc |= make_map_3d(&P.cd, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, P.d, g.nx, g.ny, g.nz, dims.tx, dims.ty, 1);
        rc |= make_map_3d(&P.cz, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, P.z, g.nx, g.ny, g.nz, dims.tx, dims.ty, 1);
        if (rc) return GBPCG_ERR_CUDA;
        P.op = make_op_const(g.nx, g.ny, g.nz);
        P.nx = g.nx; P.ny = g.ny; P.nz = g.nz;
        P.tiles_x = pg.tiles_x; P.tiles = pg.tiles;
        P.row0_item = nrow; P.nrow_items = pg.nrow_items; P.rows_per_item = pg.rows_per_item;
        if ((size_t)pg.nrow_items * 3 > 4 * kMaxPassBlocks)
            return fail_arg("persistent batch: a grid has more row items than its partial-sum slots");
        for (int k = 0; k < pg.nrow_items; ++k) row_prob.push_back(i);
        nrow += pg.nrow_items;
        auto cc = [](int m) { double h = 1.0 / (m + 1); return 1.0 / (h * h); };
        Res64Args &ra = P.ra;
        memset(&ra, 0, sizeof(ra));
        ra.nx = g.nx; ra.ny = g.ny; ra.nz = g.nz;
        ra.x = c.x; ra.b = c.b; ra.z = P.z; ra.d = P.d;
        ra.cx = cc(g.nx); ra.cy = cc(g.ny); ra.cz = cc(g.nz);
        ra.kb = nullptr; ra.kbx = ra.kby = ra.kbz = 1;
        ra.tab64 = nullptr;
        ra.bscale = nullptr;
        ra.rhs_auto = 1;
        ra.st = P.st;
        ra.partials = P.partials;
    }
    BatchHeader *hdr = reinterpret_cast<BatchHeader *>(region + BL.hdr);
    BatchProblem *dprobs = reinterpret_cast<BatchProblem *>(region + BL.probs);
    int *drows = reinterpret_cast<int *>(region + BL.rows);

    const BatchKernel K = io == GBPCG_F64 ? batch_kernel_for<double>(cfg) : batch_kernel_for<float>(cfg);
    GB_CUDA(cudaFuncSetAttribute(K.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K.smem));
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, K.fn, kBatchThreads, K.smem));
    if (occ < 1) return fail_arg("persistent batch kernel does not fit an SM");
    const unsigned grid = (unsigned)(occ * device_sm_count());

    BatchArgs A;
    A.probs = dprobs;
    A.ctl = reinterpret_cast<ProbCtl *>(region + BL.ctl);
    A.row_prob = drows;
    A.hdr = hdr;
    A.nprob = nprob;
    A.nrow_items = nrow;
    A.tol = tol;
    A.maxit = maxit;
    {
        long long tp = 0;
        for (int i = 0; i < nprob; ++i) tp += (long long)probs[i].tiles * probs[i].nz;
        A.depth0 = (int)std::max(4LL, std::min((long long)kBatchZDepth, (tp + 2LL * grid - 1) / (2LL * grid)));
    }

    // the table is copied on every call (the stream orders it before the kernel); its contents
    // depend only on the key, so a cached graph stays valid
    GB_CUDA(cudaMemcpyAsync(dprobs, probs.data(), sizeof(BatchProblem) * nprob, cudaMemcpyHostToDevice, s));
    GB_CUDA(cudaMemcpyAsync(drows, row_prob.data(), sizeof(int) * row_prob.size(), cudaMemcpyHostToDevice, s));
    GB_CUDA(cudaMemsetAsync(hdr, 0, sizeof(BatchHeader), s));
    // the host arrays must outlive the copies
    GB_CUDA(cudaStreamSynchronize(s));

    void *kargs[] = {&A};
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(kBatchThreads);
    lc.dynamicSmemBytes = K.smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;

    PersistKey key;
    key.cfg = cfg;
    key.keys.resize(nprob);
    for (int i = 0; i < nprob; ++i) key.keys[i] = make_key<float>(calls[i], true);
    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_persist_mu);
        for (auto it = g_persist.begin(); it != g_persist.end(); ++it)
            if (same_key(it->key, key)) {
                g_persist.splice(g_persist.begin(), g_persist, it);
                exec = g_persist.front().exec;
                break;
            }
        if (!exec) {
            cudaStream_t cs = nullptr;
            GB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            lc.stream = cs;
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (!e) {
                cudaError_t e2 = cudaLaunchKernelExC(&lc, K.fn, kargs);
                cudaError_t e3 = cudaStreamEndCapture(cs, &graph);
                e = e2 ? e2 : e3;
            }
            cudaGraphExec_t ex = nullptr;
            if (!e) e = cudaGraphInstantiate(&ex, graph, 0);
            cudaStreamDestroy(cs);
            lc.stream = s;
            if (e) {
                // cooperative launches that cannot be captured run directly
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
            } else {
                PersistGraph pg;
                pg.key = key;
                pg.graph = graph;
                pg.exec = ex;
                g_persist.push_front(pg);
                while (g_persist.size() > kPersistMax) {
                    cudaGraphExecDestroy(g_persist.back().exec);
                    cudaGraphDestroy(g_persist.back().graph);
                    g_persist.pop_back();
                }
                exec = ex;
            }
        }
    }
    if (exec) GB_CUDA(cudaGraphLaunch(exec, s));
    else GB_CUDA(cudaLaunchKernelExC(&lc, K.fn, kargs));
    return GBPCG_OK;
}

// Rounds run and whether a bounded barrier wait gave up, from the batch
// region (enqueued on s; valid after it synchronises).
int batch_persistent_header(const char *region, int *abort_phases, cudaStream_t s) {
    GB_CUDA(cudaMemcpyAsync(abort_phases, region + offsetof(BatchHeader, abort), 2 * sizeof(int),
                            cudaMemcpyDeviceToHost, s));
    return GBPCG_OK;
}

}  // namespace gb
