// C ABI of the iterative-refinement library: argument checking, workspace,
// the blocked LU driver and the refinement loop (Algorithm IR, Sec. 1) with the
// termination rules of Sec. 5.1.
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <new>
#include <vector>

#include "ir_internal.cuh"

namespace ir {
static std::atomic<unsigned long long> g_launch_count{0};
void count_launch() { g_launch_count.fetch_add(1, std::memory_order_relaxed); }
void count_launches(unsigned long long k) { g_launch_count.fetch_add(k, std::memory_order_relaxed); }
unsigned long long launches() { return g_launch_count.load(std::memory_order_relaxed); }
}  // namespace ir

using namespace ir;

namespace {

// Optional per-launcher timing: a pair of CUDA events around every launcher
// call on the launching stream, summed per kind when profiling stops.
enum Kind {
    KC_CAST, KC_MAXABS, KC_IOTA, KC_PANEL, KC_LASWP, KC_TRSM, KC_GEMM_SIMT, KC_GEMM_TC,
    KC_DIAGINV, KC_INIT, KC_TRSV, KC_RESID, KC_STOREX, KC_BATCHED, KC_GM_ORTH, KC_GM_UPDATE, KC_NORM1, KC_BI_STEP,
    KC_GEMM_TC_GROUP, KC_PACK, KC_TRSV64, KC_STORE, KC_U12_GROUP, KC_TERM, KC_N
};
const char *kKindNames[KC_N] = {"cast", "maxabs", "iota", "panel", "laswp", "trsm", "gemm_simt",
                                "gemm_tc", "diag_inv", "init_rb", "trsv_pair", "residual", "store_x",
                                "batched", "gm_orth", "krylov_update", "norm1", "bi_step",
                                "gemm_tc_group", "pack", "trsv_pair_f64", "store_tf", "u12_group", "term"};
struct ProfRec {
    int kind;
    cudaEvent_t a, b;
};
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<ProfRec> recs;
    cudaEvent_t next() {
        if (used == pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool.push_back(e);
        }
        return pool[used++];
    }
};
Profiler g_prof;

struct ProfScope {
    ProfRec r{};
    cudaStream_t s;
    bool active;
    ProfScope(int kind, cudaStream_t st) : s(st), active(g_prof.on) {
        if (!active) return;
        r.kind = kind;
        r.a = g_prof.next();
        r.b = g_prof.next();
        active = r.a && r.b;
        if (active) cudaEventRecord(r.a, s);
    }
    void done() {
        if (!active) return;
        cudaEventRecord(r.b, s);
        g_prof.recs.push_back(r);
    }
};

thread_local char g_last_error[256] = "";

ir_status cuda_fail(cudaError_t e, const char *what) {
    snprintf(g_last_error, sizeof g_last_error, "%s: %s", what, cudaGetErrorString(e));
    return (e == cudaErrorMemoryAllocation) ? IR_ENOMEM : IR_ECUDA;
}

#define CK(call)                                                \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
    } while (0)

// Launcher call with optional timing.
#define RUN(kind, s, call)                \
    do {                                  \
        ProfScope ps_((kind), (s));       \
        CK(call);                         \
        ps_.done();                       \
    } while (0)

constexpr int kInfoNone = 0x7F7F7F7F;   // memset(0x7F) pattern: no zero pivot
constexpr int kSwapListInts = 1 + 4 * kPanelNB;
constexpr int kPanelReserveSMs = 16;     // SMs the trailing update leaves to the next panel
constexpr int kDefaultGroup = 8;         // block steps per group of the tensor-core LU (K = 512 far updates)

bool tw_ok(ir_dtype t) { return t == IR_F64 || t == IR_F32; }
bool tf_ok(ir_dtype t) { return t == IR_F32 || t == IR_TF32 || t == IR_BF16 || t == IR_F16; }
size_t op_elem(ir_dtype tf) { return tf == IR_TF32 ? 4 : 2; }
double eps_of(ir_dtype tw) { return tw == IR_F64 ? std::ldexp(1.0, -52) : std::ldexp(1.0, -23); }

double bits_to_double(unsigned long long b) {
    double d;
    std::memcpy(&d, &b, sizeof d);
    return d;
}

ir_status ensure_partials(ir_ctx *ctx, int64_t n) {
    const int64_t need = residual_partials_needed(n, ctx->sms);
    if (need <= ctx->partials_cap) return IR_OK;
    if (ctx->partials) cudaFree(ctx->partials);
    ctx->partials = nullptr;
    ctx->partials_cap = 0;
    CK(cudaMalloc(&ctx->partials, need * sizeof(double)));
    ctx->partials_cap = need;
    return IR_OK;
}

void free_fact(ir_fact *f);

// ir_solve_host's cached buffers and factorization.
void release_host_cache(ir_ctx *ctx) {
    if (ctx->host_f) free_fact(ctx->host_f);
    ctx->host_f = nullptr;
    cudaFree(ctx->host_dA);
    cudaFree(ctx->host_db);
    cudaFree(ctx->host_dx);
    ctx->host_dA = ctx->host_db = ctx->host_dx = nullptr;
    ctx->host_n = -1;
}

void free_fact(ir_fact *f) {
    if (!f) return;
    cudaFree(f->AF);
    cudaFree(f->ipiv);
    cudaFree(f->perm);
    cudaFree(f->swap_list);
    cudaFree(f->Aop);
    cudaFree(f->Bop);
    cudaFree(f->Agrp);
    cudaFree(f->Bgrp);
    cudaFree(f->y64);
    cudaFree(f->z64);
    cudaFree(f->mps_flags);
    cudaFree(f->AF16);
    cudaFree(f->xm);
    cudaFree(f->rm);
    cudaFree(f->bm);
    cudaFree(f->mtags);
    cudaFree(f->mscal);
    if (f->host_mscal) cudaFreeHost(f->host_mscal);
    cudaFree(f->Linv);
    cudaFree(f->Uinv);
    cudaFree(f->tags);
    cudaFree(f->blk_subst);
    cudaFree(f->x);
    cudaFree(f->r);
    cudaFree(f->dev);
    if (f->host_dev) cudaFreeHost(f->host_dev);
    cudaFree(f->loop);
    cudaFree(f->panel_grec);
    cudaFree(f->panel_gcnt);
    if (f->host_loop) cudaFreeHost(f->host_loop);
    cudaFree(f->gm_V);
    cudaFree(f->gm_W);
    cudaFree(f->gm_st);
    cudaFree(f->bi_V);
    cudaFree(f->bi_st);
    if (f->gm_host_k) cudaFreeHost(f->gm_host_k);
    if (f->graph) cudaGraphExecDestroy(f->graph);
    if (f->cap_stream) cudaStreamDestroy(f->cap_stream);
    if (f->la_stream) cudaStreamDestroy(f->la_stream);
    for (int i = 0; i < f->la_nevents; ++i) cudaEventDestroy(f->la_events[i]);
    delete[] f->la_events;
    delete f;
}

ir_status alloc_fact(ir_ctx *ctx, int64_t n, const ir_opts *o, ir_fact **out) {
    ir_fact *f = new (std::nothrow) ir_fact();
    if (!f) return IR_ENOMEM;
    f->ctx = ctx;
    f->n = n;
    f->TW = o->TW;
    f->TF = o->TF;
    f->TR = o->TR;
    f->fp16_scale = o->fp16_scale;
    f->nb = kPanelNB;
    f->reserve_sms = kPanelReserveSMs;
    f->group = kDefaultGroup;
    f->ldf = ((n > 0 ? n : 1) + 31) / 32 * 32;
    const int64_t nn = n > 0 ? n : 1;
    const int64_t nblk = (nn + kTrsvB - 1) / kTrsvB;
    ir_status st = IR_OK;
#define AL(ptr, bytes)                                                        \
    do {                                                                      \
        cudaError_t e_ = cudaMalloc((void **)&(ptr), (bytes));                \
        if (e_ != cudaSuccess) { st = cuda_fail(e_, "cudaMalloc"); goto fail; } \
    } while (0)
    AL(f->AF, (size_t)nn * f->ldf * sizeof(float));
    AL(f->ipiv, nn * sizeof(int32_t));
    AL(f->perm, nn * sizeof(int32_t));
    AL(f->swap_list, 2 * kMaxGroup * kSwapListInts * sizeof(int32_t));
    if (o->TF != IR_F32) {
        AL(f->Aop, 2 * (size_t)nn * kPanelNB * op_elem(o->TF));
        AL(f->Bop, 2 * (size_t)nn * kPanelNB * op_elem(o->TF));
        if (nn > 2 * kPanelNB) {
            AL(f->Agrp, (size_t)kMaxGroup * nn * kPanelNB * op_elem(o->TF));
            AL(f->Bgrp, (size_t)kMaxGroup * nn * kPanelNB * op_elem(o->TF));
        }
    }
    AL(f->Linv, (size_t)nblk * kTrsvB * kTrsvB * sizeof(float));
    AL(f->Uinv, (size_t)nblk * kTrsvB * kTrsvB * sizeof(float));
    AL(f->tags, (size_t)2 * nblk * kTrsvB * sizeof(unsigned long long));
    AL(f->blk_subst, (size_t)2 * nblk * sizeof(int32_t));
    f->onthefly = o->onthefly;
    f->store_tf = o->store_tf;
    if (o->store_tf) AL(f->AF16, (size_t)nn * f->ldf * 2);
    if (o->onthefly && o->TW == IR_F64) {
        // the mixed precision solves run in blocks of kMpsB rows
        const int64_t mblk = (nn + kMpsB - 1) / kMpsB;
        AL(f->y64, (size_t)mblk * kMpsB * sizeof(double));
        AL(f->z64, (size_t)mblk * kMpsB * sizeof(double));
        AL(f->mps_flags, (size_t)2 * mblk * sizeof(int));
        if (cudaMemset(f->mps_flags, 0, (size_t)2 * mblk * sizeof(int)) != cudaSuccess) {
            st = IR_ECUDA;
            goto fail;
        }
    }
    AL(f->x, nn * sizeof(double));
    AL(f->r, nn * sizeof(double));
    AL(f->dev, sizeof(DevScalars));
    AL(f->loop, sizeof(SolveLoop));
    if (nn > (int64_t)kPanelRows * kPanelMaxCluster) {
        AL(f->panel_grec, (size_t)2 * kPanelMaxGrid * kPanelGridRec * sizeof(float));
        AL(f->panel_gcnt, (size_t)kPanelGridCounters * sizeof(unsigned));
    }
#undef AL
    if (cudaMallocHost((void **)&f->host_dev, sizeof(DevScalars)) != cudaSuccess ||
        cudaMallocHost((void **)&f->host_loop, sizeof(SolveLoop)) != cudaSuccess) {
        st = IR_ENOMEM;
        goto fail;
    }
    if (cudaMemset(f->AF, 0, (size_t)nn * f->ldf * sizeof(float)) != cudaSuccess ||
        cudaMemset(f->tags, 0, (size_t)2 * nblk * kTrsvB * sizeof(unsigned long long)) != cudaSuccess) {
        st = IR_ECUDA;
        goto fail;
    }
    st = ensure_partials(ctx, nn);
    if (st != IR_OK) goto fail;
    f->epoch = 0;
    *out = f;
    return IR_OK;
fail:
    free_fact(f);
    return st;
}

bool lookahead_enabled() {
    const char *e = std::getenv("IR_NO_LOOKAHEAD");
    return !(e && e[0] && e[0] != '0');
}

ir_status ensure_lookahead(ir_fact *f) {
    const int need = 2 * (int)((f->n + kPanelNB - 1) / kPanelNB) + 3;
    if (!f->la_stream) {
        int lo = 0, hi = 0;
        CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        CK(cudaStreamCreateWithPriority(&f->la_stream, cudaStreamNonBlocking, lo));
    }
    if (f->la_nevents < need) {
        for (int i = 0; i < f->la_nevents; ++i) cudaEventDestroy(f->la_events[i]);
        delete[] f->la_events;
        f->la_events = new (std::nothrow) cudaEvent_t[need];
        f->la_nevents = 0;
        if (!f->la_events) return IR_ENOMEM;
        for (int i = 0; i < need; ++i) {
            CK(cudaEventCreateWithFlags(&f->la_events[i], cudaEventDisableTiming));
            f->la_nevents = i + 1;
        }
    }
    return IR_OK;
}

// Cast + blocked right-looking LU with partial pivoting + diagonal-block inverses.
//
// With lookahead (two streams, captured into one graph): step j runs
//   s1: panel(j), [wait R(j-1)], row interchanges, U12 and update of the next
//       block column only, then panel(j+1) ...
//   s2: [wait P(j)] row interchanges of the other columns, U12 and update of
//       the remaining trailing columns (persistent kernels that leave SMs to
//       the panel), record R(j)
// so the next panel overlaps the bulk of the trailing update.  The swap list
// and the tensor-core operand buffers alternate between two copies by step
// parity.  Every element still receives its updates in block order.
// Tensor-core factorization (TF = TF32, bf16, fp16) in groups of G block steps.
// Within a group the steps run as in enqueue_factor, but each step updates
// only the near columns: the rest of its group and the first block column of
// the next group.  At the group's end the far columns (everything right of
// that) receive the whole group at once:
//   1. the group's row interchanges, in order;
//   2. rTF of the group's L columns is packed into G operand slots;
//   3. U12 of the group's rows: for each of its 64-row blocks t, the binary32
//      U12 solve (writing rTF(U) into slot t), then the tensor-core update of
//      the group's rows below block t by slot t (K = 64) -- the block steps of
//      the right-looking LU, restricted to the group's rows;
//   4. the rows below the group minus the products of all G slots (K = 64 G):
//      one read and one write of each binary32 C tile for the whole group.
// Every element still receives the same TF-rounded operand products, block by
// block in order; only the binary32 accumulation of a group's products for the
// far rows is one sum instead of G.
// With lookahead (second stream s2): step 4 for the next group's near columns
// runs at the group's end, the rest of step 4 (the far columns beyond the next
// group) in G column chunks, one after each step of the next group, so the
// next group's panels overlap it.
ir_status enqueue_factor_grouped(ir_fact *f, cudaStream_t s) {
    const int n = (int)f->n;
    const int64_t ldf = f->ldf;
    CK(cudaMemsetAsync(f->dev, 0, sizeof(DevScalars), s));
    CK(cudaMemsetAsync(&f->dev->info, 0x7F, sizeof(int), s));
    if (n == 0) return IR_OK;
    const int use_scale = (f->TF == IR_F16 && f->fp16_scale) ? 1 : 0;
    if (use_scale) RUN(KC_MAXABS, s, launch_maxabs(n, f->TW, f->A, f->lda, f->dev, f->ctx->sms, s));
    RUN(KC_CAST, s, launch_cast(n, f->TW, f->A, f->lda, f->TF, use_scale, f->AF, ldf, f->dev, s));
    RUN(KC_IOTA, s, launch_iota(n, f->perm, s));
    const int NB = kPanelNB;
    const int G = f->group;
    const int W = NB * G;
    const int sms = f->ctx->sms;
    const size_t esz = op_elem(f->TF);
    const size_t opsz = (size_t)n * NB * esz;
    const bool la = !g_prof.on && lookahead_enabled() && n > 2 * NB;
    const int share = sms - f->reserve_sms;
    cudaStream_t s2 = s;
    int ev = 0;
    if (la) {
        ir_status st = ensure_lookahead(f);
        if (st != IR_OK) return st;
        s2 = f->la_stream;
        CK(cudaEventRecord(f->la_events[ev], s));       // s2 joins after the cast
        CK(cudaStreamWaitEvent(s2, f->la_events[ev], 0));
        ++ev;
    }
    // the far update of the previous group still owed to the columns [pend_cb, n)
    // (lookahead): Gp slots, column chunks of pend_w, pend_k of them enqueued
    int pend_c0 = 0, pend_G = 0, pend_cb = n, pend_w = 0, pend_near = 0;
    auto pend_chunk = [&](cudaStream_t st) -> ir_status {
        if (pend_cb >= n) return IR_OK;
        const int ce = (pend_cb + pend_w < n) ? pend_cb + pend_w : n;
        RUN(KC_GEMM_TC_GROUP, st, launch_gemm_tc_group(f->AF, ldf, pend_c0, pend_G, pend_c0 + NB * pend_G, n, pend_cb,
                                                       ce, 0, pend_G, f->TF, f->Agrp, n - pend_c0, f->Bgrp,
                                                       n - pend_near, pend_near, sms, la ? share : 0, f->dev, st));
        pend_cb = ce;
        return IR_OK;
    };
    cudaEvent_t pending_rest = nullptr;                  // R(j-1): s2's work of the previous step
    for (int c0 = 0, step = 0; c0 < n; c0 += W) {
        const int c1 = (c0 + W < n) ? c0 + W : n;
        const int near_end = (c1 + NB < n) ? c1 + NB : n;
        const int Gg = (c1 - c0 + NB - 1) / NB;
        for (int j = c0; j < c1; j += NB, ++step) {
            const int nbp = (n - j < NB) ? n - j : NB;
            const int par = step & 1;
            int32_t *sl = f->swap_list + (step % (2 * kMaxGroup)) * kSwapListInts;
            void *aop = static_cast<char *>(f->Aop) + par * opsz;
            void *bop = static_cast<char *>(f->Bop) + par * opsz;
            RUN(KC_PANEL, s, launch_panel(f->AF, ldf, n, j, nbp, f->ipiv, f->perm, sl, f->dev, f->TF, aop, s,
                                          f->panel_grec, f->panel_gcnt));
            const bool trailing = j + nbp < n;
            const bool group_end = (j + NB >= c1) && near_end < n;   // far columns get the group's update now
            cudaStream_t sw = s;                                     // stream of this step's rest
            if (la) {
                cudaEvent_t evP = f->la_events[ev++];
                CK(cudaEventRecord(evP, s));
                if (pending_rest) CK(cudaStreamWaitEvent(s, pending_rest, 0));
                pending_rest = nullptr;
                if (!trailing) {
                    RUN(KC_LASWP, s, launch_laswp(f->AF, ldf, 0, j, 0, 0, sl, s));
                    break;
                }
                const int nx0 = j + NB, nx1 = (j + 2 * NB < n) ? j + 2 * NB : n;
                // s1: the next block column
                RUN(KC_TRSM, s, launch_laswp_trsm(f->AF, ldf, nx0, nx1, j, f->TF, bop, sl, s));
                RUN(KC_GEMM_TC, s, launch_gemm_tc(f->AF, ldf, n, j, NB, nx0, nx1, f->TF, aop, bop, sms, 0, f->dev, s));
                // s2: the rest of the near columns
                CK(cudaStreamWaitEvent(s2, evP, 0));
                sw = s2;
                RUN(KC_LASWP, s2, launch_laswp(f->AF, ldf, 0, j, nx1, near_end, sl, s2));
                if (nx1 < near_end) {
                    RUN(KC_TRSM, s2, launch_trsm(f->AF, ldf, nx1, near_end, j, f->TF, bop, s2));
                    RUN(KC_GEMM_TC, s2, launch_gemm_tc(f->AF, ldf, n, j, NB, nx1, near_end, f->TF, aop, bop, sms,
                                                       share, f->dev, s2));
                }
                // one chunk of the previous group's far update
                ir_status st = pend_chunk(s2);
                if (st != IR_OK) return st;
            } else {
                RUN(KC_LASWP, s, launch_laswp(f->AF, ldf, 0, j, j + nbp, near_end, sl, s));
                if (trailing && j + NB < near_end) {
                    RUN(KC_TRSM, s, launch_trsm(f->AF, ldf, j + NB, near_end, j, f->TF, bop, s));
                    RUN(KC_GEMM_TC, s, launch_gemm_tc(f->AF, ldf, n, j, NB, j + NB, near_end, f->TF, aop, bop, sms, 0,
                                                      f->dev, s));
                }
            }
            if (group_end) {
                // the rest of the previous group's far update comes first (same columns)
                while (pend_cb < n) {
                    ir_status st = pend_chunk(sw);
                    if (st != IR_OK) return st;
                }
                const int mshare = la ? share : 0;
                // 1. the group's interchanges on the far columns, in order
                RUN(KC_LASWP, sw, launch_laswp_lists(f->AF, ldf, near_end, n, f->swap_list, kSwapListInts,
                                                     2 * kMaxGroup, step - (Gg - 1), Gg, sw));
                // 2. rTF of the group's L columns (rows below each block's diagonal block)
                RUN(KC_PACK, sw, launch_pack_slots(f->AF, ldf, c0, Gg, c0 + NB, n, n - c0, f->TF, f->Agrp, sms, sw));
                // 3. U12 of the group's rows, block by block, with the group's own block steps
                //    between them (one kernel, one CTA per 64 far columns)
                RUN(KC_U12_GROUP, sw, launch_u12_group_tc(f->AF, ldf, c0, Gg, near_end, n, f->TF, f->Agrp, n - c0,
                                                          f->Bgrp, n - near_end, near_end, f->dev, sw));
                // 4. the rows below the group: all G slots at once
                pend_c0 = c0;
                pend_G = Gg;
                pend_near = near_end;
                pend_cb = near_end;
                if (la) {
                    // now the next group's near columns; the rest in chunks during the next group
                    const int c2 = (c1 + W < n) ? c1 + W : n;
                    const int nend2 = (c2 + NB < n) ? c2 + NB : n;
                    pend_w = nend2 - near_end;
                    ir_status st = pend_chunk(sw);
                    if (st != IR_OK) return st;
                    const int steps2 = (c2 - c1 + NB - 1) / NB;
                    pend_w = ((n - pend_cb) + steps2 - 1) / steps2;
                    pend_w = (pend_w + NB - 1) / NB * NB;
                } else {
                    pend_w = n - near_end;
                    ir_status st = pend_chunk(sw);
                    if (st != IR_OK) return st;
                }
            }
            if (la) {
                pending_rest = f->la_events[ev++];
                CK(cudaEventRecord(pending_rest, s2));
            }
        }
    }
    if (pend_cb < n) {
        // chunks the last group had no steps left for (not expected; kept for safety)
        cudaStream_t st = la ? s2 : s;
        while (pend_cb < n) {
            ir_status e = pend_chunk(st);
            if (e != IR_OK) return e;
        }
        if (la) {
            pending_rest = f->la_events[ev++];
            CK(cudaEventRecord(pending_rest, s2));
        }
    }
    if (pending_rest) CK(cudaStreamWaitEvent(s, pending_rest, 0));
    if (f->store_tf) RUN(KC_STORE, s, launch_store_tf(f->AF, ldf, n, f->TF, f->AF16, f->dev, sms, s));
    RUN(KC_DIAGINV, s, launch_diag_inv(f->AF, ldf, n, f->Linv, f->Uinv, f->blk_subst, s));
    return IR_OK;
}

ir_status enqueue_factor(ir_fact *f, cudaStream_t s) {
    if (f->TF != IR_F32 && f->Agrp) return enqueue_factor_grouped(f, s);
    const int n = (int)f->n;
    const int64_t ldf = f->ldf;
    CK(cudaMemsetAsync(f->dev, 0, sizeof(DevScalars), s));
    CK(cudaMemsetAsync(&f->dev->info, 0x7F, sizeof(int), s));
    if (n == 0) return IR_OK;
    const int use_scale = (f->TF == IR_F16 && f->fp16_scale) ? 1 : 0;
    if (use_scale) RUN(KC_MAXABS, s, launch_maxabs(n, f->TW, f->A, f->lda, f->dev, f->ctx->sms, s));
    RUN(KC_CAST, s, launch_cast(n, f->TW, f->A, f->lda, f->TF, use_scale, f->AF, ldf, f->dev, s));
    RUN(KC_IOTA, s, launch_iota(n, f->perm, s));
    const int NB = kPanelNB;
    const int sms = f->ctx->sms;
    const size_t opsz = (f->TF == IR_F32) ? 0 : (size_t)n * NB * op_elem(f->TF);
    const bool la = !g_prof.on && lookahead_enabled() && n > 2 * NB;
    cudaStream_t s2 = s;
    int ev = 0;
    if (la) {
        ir_status st = ensure_lookahead(f);
        if (st != IR_OK) return st;
        s2 = f->la_stream;
        CK(cudaEventRecord(f->la_events[ev], s));       // s2 joins after the cast
        CK(cudaStreamWaitEvent(s2, f->la_events[ev], 0));
        ++ev;
    }
    cudaEvent_t pending_rest = nullptr;                  // R(j-1): s2's work of the previous step
    for (int j = 0, step = 0; j < n; j += NB, ++step) {
        const int nbp = (n - j < NB) ? n - j : NB;
        const int par = step & 1;
        int32_t *sl = f->swap_list + par * kSwapListInts;
        void *aop = f->Aop ? static_cast<char *>(f->Aop) + par * opsz : nullptr;
        void *bop = f->Bop ? static_cast<char *>(f->Bop) + par * opsz : nullptr;
        RUN(KC_PANEL, s, launch_panel(f->AF, ldf, n, j, nbp, f->ipiv, f->perm, sl, f->dev, f->TF, aop, s,
                                          f->panel_grec, f->panel_gcnt));
        const bool trailing = j + nbp < n;
        if (la) {
            cudaEvent_t evP = f->la_events[ev++];
            CK(cudaEventRecord(evP, s));
            if (pending_rest) CK(cudaStreamWaitEvent(s, pending_rest, 0));
            pending_rest = nullptr;
            if (!trailing) {
                RUN(KC_LASWP, s, launch_laswp(f->AF, ldf, 0, j, 0, 0, sl, s));
                break;
            }
            const int nx0 = j + NB, nx1 = (j + 2 * NB < n) ? j + 2 * NB : n;
            // s1: the next block column
            RUN(KC_TRSM, s, launch_laswp_trsm(f->AF, ldf, nx0, nx1, j, f->TF, bop, sl, s));
            if (f->TF == IR_F32)
                RUN(KC_GEMM_SIMT, s, launch_gemm_simt(f->AF, ldf, n, j, NB, nx0, nx1, 0, s));
            else
                RUN(KC_GEMM_TC, s, launch_gemm_tc(f->AF, ldf, n, j, NB, nx0, nx1, f->TF, aop, bop, sms, 0, f->dev, s));
            // s2: everything else of this step
            CK(cudaStreamWaitEvent(s2, evP, 0));
            RUN(KC_LASWP, s2, launch_laswp(f->AF, ldf, 0, j, nx1, n, sl, s2));
            if (nx1 < n) {
                RUN(KC_TRSM, s2, launch_trsm(f->AF, ldf, nx1, n, j, f->TF, bop, s2));
                if (f->TF == IR_F32)
                    RUN(KC_GEMM_SIMT, s2, launch_gemm_simt(f->AF, ldf, n, j, NB, nx1, n, sms - f->reserve_sms, s2));
                else
                    RUN(KC_GEMM_TC, s2, launch_gemm_tc(f->AF, ldf, n, j, NB, nx1, n, f->TF, aop, bop, sms,
                                                       sms - f->reserve_sms, f->dev, s2));
            }
            pending_rest = f->la_events[ev++];
            CK(cudaEventRecord(pending_rest, s2));
        } else {
            RUN(KC_LASWP, s, launch_laswp(f->AF, ldf, 0, j, j + nbp, n, sl, s));
            if (trailing) {
                RUN(KC_TRSM, s, launch_trsm(f->AF, ldf, j + NB, n, j, f->TF, bop, s));
                if (f->TF == IR_F32)
                    RUN(KC_GEMM_SIMT, s, launch_gemm_simt(f->AF, ldf, n, j, NB, j + NB, n, 0, s));
                else
                    RUN(KC_GEMM_TC, s, launch_gemm_tc(f->AF, ldf, n, j, NB, j + NB, n, f->TF, aop, bop, sms, 0,
                                                      f->dev, s));
            }
        }
    }
    if (pending_rest) CK(cudaStreamWaitEvent(s, pending_rest, 0));
    if (f->store_tf) RUN(KC_STORE, s, launch_store_tf(f->AF, ldf, n, f->TF, f->AF16, f->dev, sms, s));
    RUN(KC_DIAGINV, s, launch_diag_inv(f->AF, ldf, n, f->Linv, f->Uinv, f->blk_subst, s));
    return IR_OK;
}

bool graphs_enabled() {
    const char *e = std::getenv("IR_NO_GRAPH");
    return !(e && e[0] && e[0] != '0');
}

// The factorization's launch sequence is captured once per (A, lda) into a
// CUDA graph on a private stream and replayed on the caller's stream; with
// per-launcher profiling on, the launches are issued directly instead.
ir_status run_factor(ir_fact *f, cudaStream_t s) {
    // a factorization with cooperative panels (n > 8192) is enqueued directly
    if (g_prof.on || !graphs_enabled() || f->n == 0 || f->panel_grec) return enqueue_factor(f, s);
    if (!f->graph || f->graph_A != f->A || f->graph_lda != f->lda) {
        if (f->graph) {
            cudaGraphExecDestroy(f->graph);
            f->graph = nullptr;
        }
        if (!f->cap_stream) CK(cudaStreamCreateWithFlags(&f->cap_stream, cudaStreamNonBlocking));
        const unsigned long long l0 = ir::launches();
        CK(cudaStreamBeginCapture(f->cap_stream, cudaStreamCaptureModeThreadLocal));
        ir_status st = enqueue_factor(f, f->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(f->cap_stream, &g);
        if (st != IR_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&f->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            f->graph = nullptr;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        f->graph_launches = ir::launches() - l0;
        g_launch_count.fetch_sub(f->graph_launches, std::memory_order_relaxed);  // captured, not run
        f->graph_A = f->A;
        f->graph_lda = f->lda;
    }
    CK(cudaGraphLaunch(f->graph, s));
    ir::count_launches(f->graph_launches);
    return IR_OK;
}

ir_status read_dev(ir_fact *f, cudaStream_t s) {
    CK(cudaMemcpyAsync(f->host_dev, f->dev, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return IR_OK;
}

// Termination test of Sec. 5.1 after the k-th residual (the rule shared with
// the device loop, ir_internal.cuh): -1 to continue, else an ir_solve_status.
int term_decide(const double *rh, const double *dh, int k, double bnorm, double eps_w,
                const ir_term *t, bool tr_wider, double rmax_r, double anorm, double xnorm) {
    TermArgs ta;
    ta.Cr = t->Cr;
    ta.Ce = t->Ce;
    ta.Rmax = t->Rmax;
    ta.rmax_r = rmax_r;
    ta.abs_rel_tol = t->abs_rel_tol;
    ta.eps_w = eps_w;
    ta.litmax = t->litmax;
    ta.mode = t->mode;
    ta.tr_wider = tr_wider ? 1 : 0;
    return term_rule(rh, dh, k, bnorm, ta, anorm, xnorm);
}

}  // namespace

ir_status ir::record_cuda_error(cudaError_t e, const char *what) { return cuda_fail(e, what); }

// A planned batch (ir_batch_create): descriptors and the largest-first order on
// the device, the ticket counter of the persistent launch, the workspace slots.
struct ir_batch {
    ir_ctx *ctx;
    int64_t count;
    ir_dtype TW, TF;
    int fp16_scale;
    ir_term term;
    void *desc;          // count descriptors (device)
    int *order;          // count system indices, largest n first (device)
    unsigned *ticket;    // next position in `order` (device)
    float *ws;           // grid slots of ws_stride floats
    int64_t ws_stride;
    int grid;
    int tc_min_trail;    // smallest trailing block updated on the tensor cores (tuned)
    int *order2;         // escalation: the unconverged members (device)
    unsigned *count2;    // and their number (device)
};

namespace {

void free_batch(ir_batch *b) {
    if (!b) return;
    cudaFree(b->desc);
    cudaFree(b->order);
    cudaFree(b->order2);
    cudaFree(b->count2);
    cudaFree(b->ticket);
    cudaFree(b->ws);
    delete b;
}

}  // namespace

namespace {

// Time one replay of a planned batch (ms) on a private stream.
ir_status time_batch(ir_batch *b, ir_batch_result *res, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                     float *ms) {
    CK(cudaEventRecord(e0, s));
    CK(launch_batched(b->desc, b->order, b->count, b->ticket, b->ws, b->ws_stride, b->grid, b->TW, b->TF,
                      b->fp16_scale, &b->term, b->tc_min_trail, res, s));
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(ms, e0, e1));
    return IR_OK;
}

// Autotuner of the batched driver (opts.autotune): the smallest trailing block
// that goes to the tensor cores -- below it the CTA's SIMT update, whose setup
// is cheaper, does the same rounding-to-TF work.  Each candidate runs the
// batch itself (its A and b are only read; x is rewritten by every run) twice,
// the second timed; the fastest is kept in the plan.
ir_status tune_batch(ir_batch *b) {
    const int cands[] = {64, 128, 192, 256, 1 << 20};
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ir_batch_result *res = nullptr;
    ir_status st = IR_OK;
    float best = 3.4e38f;
    int best_c = b->tc_min_trail;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMalloc(&res, (size_t)b->count * sizeof(ir_batch_result));
    if (e != cudaSuccess) st = cuda_fail(e, "tune_batch");
    for (int c : cands) {
        if (st != IR_OK) break;
        b->tc_min_trail = c;
        float ms = 0.f;
        st = time_batch(b, res, s, e0, e1, &ms);
        if (st == IR_OK) st = time_batch(b, res, s, e0, e1, &ms);
        if (st == IR_OK && ms < best) {
            best = ms;
            best_c = c;
        }
    }
    b->tc_min_trail = best_c;
    if (res) cudaFree(res);
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (s) cudaStreamDestroy(s);
    return st;
}

// Autotuner of the single-system factorization (opts.autotune): how many SMs
// the lookahead's trailing update leaves free for the next panel's cluster.
// Each candidate factors the caller's A twice (graph captured for it), the
// second timed; the fastest is kept and remembered by the context per (n, TF).
ir_status tune_factor(ir_fact *f, cudaStream_t s) {
    ir_ctx *c = f->ctx;
    for (int i = 0; i < c->ntuned && i < 16; ++i)
        if (c->tuned[i].n == f->n && c->tuned[i].tf == (int)f->TF) {
            f->reserve_sms = c->tuned[i].reserve_sms;
            f->group = c->tuned[i].group;
            return IR_OK;
        }
    const int cands[] = {8, 12, 16, 24, 32};
    // block steps per group of the tensor-core factorization (no groups for binary32)
    const int gcands_tc[] = {4, 8, 16};
    const int gcands_f32[] = {kDefaultGroup};
    const bool tc = f->TF != IR_F32 && f->Agrp;
    const int *gc = tc ? gcands_tc : gcands_f32;
    const int ng = tc ? 3 : 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 3.4e38f;
    int best_r = f->reserve_sms, best_g = f->group;
    ir_status st = IR_OK;
    for (int gi = 0; gi < ng && st == IR_OK; ++gi)
        for (int r : cands) {
            if (r >= c->sms / 2) continue;
            f->reserve_sms = r;
            f->group = gc[gi];
            if (f->graph) {
                cudaGraphExecDestroy(f->graph);
                f->graph = nullptr;
            }
            float ms = 0.f;
            for (int rep = 0; rep < 2 && st == IR_OK; ++rep) {
                cudaError_t e = cudaEventRecord(e0, s);
                if (e == cudaSuccess) {
                    st = run_factor(f, s);
                    if (st == IR_OK) e = cudaEventRecord(e1, s);
                }
                if (st == IR_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (st == IR_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (st == IR_OK && e != cudaSuccess) st = cuda_fail(e, "tune_factor");
            }
            if (st != IR_OK) break;
            if (ms < best) {
                best = ms;
                best_r = r;
                best_g = gc[gi];
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != IR_OK) return st;
    f->reserve_sms = best_r;
    f->group = best_g;
    if (f->graph) {
        cudaGraphExecDestroy(f->graph);
        f->graph = nullptr;
    }
    ir_tuned &slot = c->tuned[c->ntuned % 16];
    slot.n = f->n;
    slot.tf = (int)f->TF;
    slot.reserve_sms = best_r;
    slot.group = best_g;
    c->ntuned += 1;
    return IR_OK;
}

}  // namespace

extern "C" {

void ir_default_opts(ir_opts *o) {
    if (!o) return;
    o->TW = IR_F64;
    o->TF = IR_F32;
    o->TR = IR_F64;
    o->fp16_scale = 1;
    o->nb = 0;
    o->autotune = 0;
    o->group = 0;
    o->onthefly = 0;
    o->store_tf = 0;
}

void ir_default_term(ir_term *t) {
    if (!t) return;
    t->Cr = 1.0;
    t->Ce = 1.0;
    t->Rmax = 0.5;
    t->litmax = 10;
    t->mode = 0;
    t->abs_rel_tol = 0.0;
}

const char *ir_last_error(void) { return g_last_error; }

unsigned long long ir_kernel_launches(void) { return ir::launches(); }

void ir_profile_start(void) {
    g_prof.on = true;
    g_prof.used = 0;
    g_prof.recs.clear();
}

int ir_profile_stop(double *ms, int *counts, int max_kinds) {
    const bool was_on = g_prof.on;
    g_prof.on = false;
    if (!was_on) return 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    for (int k = 0; k < max_kinds && k < KC_N; ++k) {
        if (ms) ms[k] = 0.0;
        if (counts) counts[k] = 0;
    }
    for (const ProfRec &r : g_prof.recs) {
        float t = 0.f;
        if (r.kind >= max_kinds || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) continue;
        if (ms) ms[r.kind] += t;
        if (counts) counts[r.kind] += 1;
    }
    g_prof.recs.clear();
    return KC_N;
}

const char *ir_profile_kind(int k) { return (k >= 0 && k < KC_N) ? kKindNames[k] : ""; }

ir_status ir_init(int device, ir_ctx **out) {
    if (!out) return IR_EINVAL;
    *out = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return IR_EINVAL;
    CK(cudaSetDevice(device));
    cudaDeviceProp p;
    CK(cudaGetDeviceProperties(&p, device));
    if (p.major != 10 || p.minor != 3) {
        snprintf(g_last_error, sizeof g_last_error, "device %d is sm_%d%d; this library is built for sm_103a",
                 device, p.major, p.minor);
        return IR_EUNSUPPORTED;
    }
    ir_ctx *c = new (std::nothrow) ir_ctx();
    if (!c) return IR_ENOMEM;
    c->device = device;
    c->sms = p.multiProcessorCount;
    c->partials = nullptr;
    c->partials_cap = 0;
    if (cudaMalloc(&c->rnorm_tmp, sizeof(double)) != cudaSuccess) {
        delete c;
        return IR_ENOMEM;
    }
    *out = c;
    return IR_OK;
}

void ir_finalize(ir_ctx *c) {
    if (!c) return;
    release_host_cache(c);
    cudaFree(c->partials);
    cudaFree(c->rnorm_tmp);
    delete c;
}

ir_status ir_factor(ir_ctx *ctx, int64_t n, const void *A, int64_t lda, const ir_opts *opts,
                    void *stream, ir_fact **out) {
    if (!ctx || !out || n < 0 || (n > 0 && !A) || lda < (n > 1 ? n : 1)) return IR_EINVAL;
    *out = nullptr;
    ir_opts o;
    if (opts) o = *opts;
    else ir_default_opts(&o);
    if (!tw_ok(o.TW) || !tf_ok(o.TF) || o.TR != IR_F64) return IR_EINVAL;
    if (o.nb != 0 && o.nb != kPanelNB) return IR_EUNSUPPORTED;
    if (o.group < 0 || o.group > kMaxGroup || (o.onthefly != 0 && o.onthefly != 1)) return IR_EINVAL;
    if (o.store_tf != 0 && (o.store_tf != 1 || (o.TF != IR_F16 && o.TF != IR_BF16))) return IR_EINVAL;
    if (n > kMaxN) {
        snprintf(g_last_error, sizeof g_last_error, "n = %lld exceeds the supported maximum %d",
                 (long long)n, kMaxN);
        return IR_EUNSUPPORTED;
    }
    CK(cudaSetDevice(ctx->device));
    ir_fact *f = nullptr;
    ir_status st = alloc_fact(ctx, n, &o, &f);
    if (st != IR_OK) return st;
    f->A = A;
    f->lda = lda;
    f->anorm_valid = 0;
    if (o.group > 0) f->group = o.group;
    // the schedule autotuner matters once the lookahead overlaps panels with updates
    if (o.autotune && n >= 1024) st = tune_factor(f, (cudaStream_t)stream);
    if (st == IR_OK) st = run_factor(f, (cudaStream_t)stream);
    if (st != IR_OK) {
        free_fact(f);
        return st;
    }
    *out = f;
    return IR_OK;
}

ir_status ir_refactor(ir_fact *f, const void *B, int64_t ldb, void *stream) {
    if (!f || (f->n > 0 && !B) || ldb < (f->n > 1 ? f->n : 1)) return IR_EINVAL;
    f->A = B;
    f->lda = ldb;
    f->anorm_valid = 0;
    return run_factor(f, (cudaStream_t)stream);
}

ir_status ir_fact_info(const ir_fact *fc, int64_t *info, int *nonfinite) {
    if (!fc) return IR_EINVAL;
    ir_fact *f = const_cast<ir_fact *>(fc);
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(f->host_dev, f->dev, sizeof(DevScalars), cudaMemcpyDeviceToHost));
    if (info) *info = f->host_dev->info == kInfoNone ? 0 : f->host_dev->info;
    if (nonfinite) *nonfinite = f->host_dev->nonfinite;
    return IR_OK;
}

ir_status ir_solve(ir_fact *f, const void *b, void *x, const ir_term *term, void *stream,
                   ir_report *rep) {
    if (!f || (f->n > 0 && (!b || !x))) return IR_EINVAL;
    ir_term t;
    if (term) t = *term;
    else ir_default_term(&t);
    if (t.litmax < 1 || t.litmax > IR_MAX_HIST - 1 || !(t.Rmax > 0) || (t.mode != 0 && t.mode != 1))
        return IR_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = f->n;
    ir_report R;
    std::memset(&R, 0, sizeof R);
    R.scale = 1.0;
    if (n == 0) {
        R.status = IR_CONVERGED;
        if (rep) *rep = R;
        return IR_OK;
    }
    CK(cudaSetDevice(f->ctx->device));
    // factorization outcome
    ir_status st = read_dev(f, s);
    if (st != IR_OK) return st;
    R.scale = f->host_dev->scale;
    if (f->host_dev->timeout) {
        snprintf(g_last_error, sizeof g_last_error, "a bounded wait in the factorization timed out");
        R.status = IR_FAILED;
        if (rep) *rep = R;
        return IR_ETIMEOUT;
    }
    if (f->host_dev->nonfinite) {
        R.status = IR_FAILED;
        if (rep) *rep = R;
        return IR_ENONFINITE;
    }
    if (f->host_dev->info != kInfoNone) {
        R.info = f->host_dev->info;
        R.status = IR_FAILED;
        if (rep) *rep = R;
        return IR_ESINGULAR;
    }
    // x = 0, r = b, rhist[0] = ||b||
    CK(cudaMemsetAsync(&f->dev->bnorm_bits, 0, sizeof(unsigned long long), s));
    RUN(KC_INIT, s, launch_init_rb(n, f->TW, b, f->r, f->x, f->dev, s));
    CK(cudaMemcpyAsync(&f->dev->rnorm_bits, &f->dev->bnorm_bits, sizeof(unsigned long long),
                       cudaMemcpyDeviceToDevice, s));
    if (t.mode == 1 && !f->anorm_valid)
        RUN(KC_NORM1, s, launch_norm1(n, f->TW, f->A, f->lda, &f->dev->anorm_bits, s));
    // The refinement loop runs on the device: litmax corrections are enqueued at
    // once, each followed by the termination test (k_loop_step); once it has
    // decided, the remaining kernels return at once.  One read-back at the end.
    TermArgs ta;
    ta.Cr = t.Cr;
    ta.Ce = t.Ce;
    ta.Rmax = t.Rmax;
    ta.rmax_r = t.Rmax;
    ta.abs_rel_tol = t.abs_rel_tol;
    ta.eps_w = eps_of(f->TW);
    ta.litmax = t.litmax;
    ta.mode = t.mode;
    ta.tr_wider = (f->TW == IR_F32) ? 1 : 0;
    const bool mps64 = f->onthefly && f->TW == IR_F64;
    if (f->onthefly && !mps64) {
        // TW = binary32: r rounded to binary32, binary32 solves with unit scale
        static const double one = 1.0;
        CK(cudaMemcpyAsync(&f->dev->one_bits, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    }
    RUN(KC_TERM, s, launch_loop_start(f->dev, f->loop, ta, s));
    const int *done = &f->loop->done;
    for (int it = 0; it < t.litmax; ++it) {
        f->epoch += 1;
        if (mps64)
            RUN(KC_TRSV64, s, launch_mps_pair(f->AF, f->ldf, (int)n, f->perm, f->r, f->x, f->y64, f->z64,
                                              f->mps_flags, f->epoch, f->dev, s, done));
        else
            RUN(KC_TRSV, s, launch_trsv_pair(f->AF, f->ldf, (int)n, f->Linv, f->Uinv, f->blk_subst, f->perm, f->r,
                                             nullptr, nullptr, f->x, f->tags, f->epoch, f->dev, s, nullptr,
                                             nullptr, done, f->onthefly != 0, f->AF16, f->TF));
        RUN(KC_RESID, s, launch_residual(n, f->TW, f->A, f->lda, b, f->x, f->r, f->ctx->partials,
                           f->ctx->partials_cap, &f->dev->rnorm_bits, f->ctx->sms, s, done));
        RUN(KC_TERM, s, launch_loop_step(f->dev, f->loop, ta, s));
    }
    // x is written unless the solve failed (b not finite, or a wait timed out)
    RUN(KC_STOREX, s, launch_store_x(n, f->TW, f->x, x, s, &f->loop->err));
    CK(cudaMemcpyAsync(f->host_loop, f->loop, sizeof(SolveLoop), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const SolveLoop &L = *f->host_loop;
    if (L.err == kLoopNonfinite) {
        // b (or A's norm) is not finite: the flag belongs to this call, not to the factorization
        CK(cudaMemsetAsync(&f->dev->nonfinite, 0, sizeof(int), s));
        R.status = IR_FAILED;
        if (rep) *rep = R;
        return IR_ENONFINITE;
    }
    if (L.err == kLoopTimeout) {
        snprintf(g_last_error, sizeof g_last_error, "a bounded wait in the triangular solve timed out");
        return IR_ETIMEOUT;
    }
    if (t.mode == 1) f->anorm_valid = 1;
    R.iters = L.k;
    R.status = (ir_solve_status)L.status;
    for (int i = 0; i <= L.k && i < IR_MAX_HIST; ++i) R.rhist[i] = L.rhist[i];
    for (int i = 0; i < L.k && i < IR_MAX_HIST; ++i) R.dhist[i] = L.dhist[i];
    if (rep) *rep = R;
    return IR_OK;
}

void ir_default_krylov_opts(ir_krylov_opts *o) {
    if (!o) return;
    o->basissize = 10;
    o->eta = 1e-8;
    o->Rmax_r = 1.0;
}

}  // extern "C"

namespace {

// The product buffer W, the pinned iteration count and the basis stride shared
// by both Krylov solvers.
ir_status krylov_common(ir_fact *f) {
    if (f->gm_W) return IR_OK;
    const int64_t n = f->n > 0 ? f->n : 1;
    f->gm_ldv = (n + 31) / 32 * 32;
    CK(cudaMalloc(&f->gm_W, (size_t)f->gm_ldv * sizeof(double)));
    if (!f->gm_host_k) CK(cudaMallocHost((void **)&f->gm_host_k, sizeof(int)));
    return IR_OK;
}

}  // namespace

extern "C" {

ir_status ir_gmres_reserve(ir_fact *f, int m) {
    if (!f || m < 1 || m > IR_MAX_BASIS) return IR_EINVAL;
    if (f->gm_st && f->gm_m >= m) return IR_OK;
    CK(cudaSetDevice(f->ctx->device));
    CK(cudaDeviceSynchronize());     // the old buffers may be in use
    ir_status st = krylov_common(f);
    if (st != IR_OK) return st;
    cudaFree(f->gm_V);
    cudaFree(f->gm_st);
    f->gm_V = nullptr;
    f->gm_st = nullptr;
    f->gm_m = 0;
    CK(cudaMalloc(&f->gm_V, (size_t)(m + 1) * f->gm_ldv * sizeof(double)));
    CK(cudaMalloc(&f->gm_st, sizeof(GmState)));
    CK(cudaMemset(f->gm_st, 0, sizeof(GmState)));
    f->gm_m = m;
    return IR_OK;
}

ir_status ir_bicgstab_reserve(ir_fact *f) {
    if (!f) return IR_EINVAL;
    if (f->bi_st) return IR_OK;
    CK(cudaSetDevice(f->ctx->device));
    ir_status st = krylov_common(f);
    if (st != IR_OK) return st;
    CK(cudaMalloc(&f->bi_V, (size_t)kBiCols * f->gm_ldv * sizeof(double)));
    CK(cudaMalloc(&f->bi_st, sizeof(BiState)));
    CK(cudaMemset(f->bi_st, 0, sizeof(BiState)));
    return IR_OK;
}

}  // extern "C"

namespace {

enum { KRY_GMRES = 0, KRY_BICGSTAB = 1 };

// Krylov-IR (Sec. 4.2-4.3): Algorithm IR with the correction equation solved by
// left-preconditioned GMRES or BiCGSTAB.
ir_status krylov_solve(int method, ir_fact *f, const void *b, void *x, const ir_term *term,
                       const ir_krylov_opts *kopts, void *stream, ir_report *rep, int *khist) {
    if (!f || (f->n > 0 && (!b || !x))) return IR_EINVAL;
    ir_term t;
    if (term) t = *term;
    else ir_default_term(&t);
    ir_krylov_opts ko;
    if (kopts) ko = *kopts;
    else ir_default_krylov_opts(&ko);
    if (t.litmax < 1 || t.litmax > IR_MAX_HIST - 1 || !(t.Rmax > 0) || (t.mode != 0 && t.mode != 1))
        return IR_EINVAL;
    if (ko.basissize < 1 || ko.basissize > IR_MAX_BASIS || !(ko.eta >= 0) || !(ko.Rmax_r > 0)) return IR_EINVAL;
    if (khist) std::memset(khist, 0, IR_MAX_HIST * sizeof(int));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = f->n;
    ir_report R;
    std::memset(&R, 0, sizeof R);
    R.scale = 1.0;
    if (n == 0) {
        R.status = IR_CONVERGED;
        if (rep) *rep = R;
        return IR_OK;
    }
    CK(cudaSetDevice(f->ctx->device));
    ir_status st = (method == KRY_GMRES) ? ir_gmres_reserve(f, ko.basissize) : ir_bicgstab_reserve(f);
    if (st != IR_OK) return st;
    st = read_dev(f, s);
    if (st != IR_OK) return st;
    R.scale = f->host_dev->scale;
    if (f->host_dev->timeout) {
        snprintf(g_last_error, sizeof g_last_error, "a bounded wait in the factorization timed out");
        R.status = IR_FAILED;
        if (rep) *rep = R;
        return IR_ETIMEOUT;
    }
    if (f->host_dev->nonfinite) {
        R.status = IR_FAILED;
        if (rep) *rep = R;
        return IR_ENONFINITE;
    }
    if (f->host_dev->info != kInfoNone) {
        R.info = f->host_dev->info;
        R.status = IR_FAILED;
        if (rep) *rep = R;
        return IR_ESINGULAR;
    }
    CK(cudaMemsetAsync(&f->dev->bnorm_bits, 0, sizeof(unsigned long long), s));
    RUN(KC_INIT, s, launch_init_rb(n, f->TW, b, f->r, f->x, f->dev, s));
    CK(cudaMemcpyAsync(&f->dev->rnorm_bits, &f->dev->bnorm_bits, sizeof(unsigned long long),
                       cudaMemcpyDeviceToDevice, s));
    if (t.mode == 1 && !f->anorm_valid)
        RUN(KC_NORM1, s, launch_norm1(n, f->TW, f->A, f->lda, &f->dev->anorm_bits, s));
    st = read_dev(f, s);
    if (st != IR_OK) return st;
    if (f->host_dev->nonfinite) {
        // b (or A's norm) is not finite: the flag belongs to this call, not to the factorization
        CK(cudaMemsetAsync(&f->dev->nonfinite, 0, sizeof(int), s));
        R.status = IR_FAILED;
        if (rep) *rep = R;
        return IR_ENONFINITE;
    }
    if (t.mode == 1) f->anorm_valid = 1;
    const double anorm = bits_to_double(f->host_dev->anorm_bits);
    const double bnorm = bits_to_double(f->host_dev->bnorm_bits);
    R.rhist[0] = bnorm;
    const bool tr_wider = (f->TW == IR_F32);
    const double eps_w = eps_of(f->TW);
    const int m = ko.basissize;
    const int nn = (int)n;
    double *V = f->gm_V, *W = f->gm_W;
    const int64_t ldv = f->gm_ldv;
    GmState *gs = f->gm_st;
    int k = 0;
    int status = (bnorm == 0.0) ? IR_CONVERGED : -1;
    double *Vb = f->bi_V;
    BiState *bs = f->bi_st;
    // w = P (A u) into out: the high-precision product, then the preconditioner;
    // both skipped once the Krylov iteration has stopped (*skip != 0)
    auto prec_matvec = [&](const double *u, double *out, unsigned long long *wbits, const int *skip) -> ir_status {
        RUN(KC_RESID, s, launch_residual(n, f->TW, f->A, f->lda, nullptr, u, W, f->ctx->partials,
                                         f->ctx->partials_cap, wbits, f->ctx->sms, s, skip));
        f->epoch += 1;
        RUN(KC_TRSV, s, launch_trsv_pair(f->AF, f->ldf, nn, f->Linv, f->Uinv, f->blk_subst, f->perm, W,
                                         nullptr, nullptr, nullptr, f->tags, f->epoch, f->dev, s, wbits, out,
                                         skip, false, f->AF16, f->TF));
        return IR_OK;
    };
    while (status < 0) {
        // z = P r
        double *z = (method == KRY_GMRES) ? V : Vb + (int64_t)kBiR * ldv;
        f->epoch += 1;
        RUN(KC_TRSV, s, launch_trsv_pair(f->AF, f->ldf, nn, f->Linv, f->Uinv, f->blk_subst, f->perm, f->r,
                                         nullptr, nullptr, nullptr, f->tags, f->epoch, f->dev, s,
                                         &f->dev->rnorm_bits, z, nullptr, false, f->AF16, f->TF));
        CK(cudaMemsetAsync(&f->dev->dnorm_bits, 0, 2 * sizeof(unsigned long long), s));   // dnorm, xnorm
        if (method == KRY_GMRES) {
            RUN(KC_GM_ORTH, s, launch_gm_orth(nn, V, ldv, -1, m, ko.eta, gs, s));     // v_0 = z / ||z||_2
            for (int j = 0; j < m; ++j) {
                st = prec_matvec(V + (int64_t)j * ldv, V + (int64_t)(j + 1) * ldv, &gs->wnorm_bits, &gs->done);
                if (st != IR_OK) return st;
                RUN(KC_GM_ORTH, s, launch_gm_orth(nn, V, ldv, j, m, ko.eta, gs, s));
            }
            RUN(KC_GM_UPDATE, s, launch_gm_update(nn, V, ldv, gs, f->x, &f->dev->dnorm_bits, &f->dev->xnorm_bits, s));
            CK(cudaMemcpyAsync(f->gm_host_k, &gs->k, sizeof(int), cudaMemcpyDeviceToHost, s));
        } else {
            RUN(KC_BI_STEP, s, launch_bi_step(0, nn, Vb, ldv, m, ko.eta, bs, s));
            for (int j = 0; j < m; ++j) {
                RUN(KC_BI_STEP, s, launch_bi_step(1, nn, Vb, ldv, m, ko.eta, bs, s));
                st = prec_matvec(Vb + (int64_t)kBiP * ldv, Vb + (int64_t)kBiV * ldv, &bs->wnorm_bits, &bs->done);
                if (st != IR_OK) return st;
                RUN(KC_BI_STEP, s, launch_bi_step(2, nn, Vb, ldv, m, ko.eta, bs, s));
                st = prec_matvec(Vb + (int64_t)kBiS * ldv, Vb + (int64_t)kBiT * ldv, &bs->wnorm_bits, &bs->done);
                if (st != IR_OK) return st;
                RUN(KC_BI_STEP, s, launch_bi_step(3, nn, Vb, ldv, m, ko.eta, bs, s));
            }
            RUN(KC_GM_UPDATE, s, launch_axpy_norms(nn, Vb + (int64_t)kBiD * ldv, f->x, &f->dev->dnorm_bits,
                                                   &f->dev->xnorm_bits, s));
            CK(cudaMemcpyAsync(f->gm_host_k, &bs->k, sizeof(int), cudaMemcpyDeviceToHost, s));
        }
        RUN(KC_RESID, s, launch_residual(n, f->TW, f->A, f->lda, b, f->x, f->r, f->ctx->partials,
                                         f->ctx->partials_cap, &f->dev->rnorm_bits, f->ctx->sms, s));
        st = read_dev(f, s);
        if (st != IR_OK) return st;
        if (f->host_dev->timeout) {
            snprintf(g_last_error, sizeof g_last_error, "a bounded wait in the triangular solve timed out");
            return IR_ETIMEOUT;
        }
        if (khist) khist[k] = *f->gm_host_k;
        ++k;
        R.dhist[k - 1] = bits_to_double(f->host_dev->dnorm_bits);
        R.rhist[k] = bits_to_double(f->host_dev->rnorm_bits);
        status = term_decide(R.rhist, R.dhist, k, bnorm, eps_w, &t, tr_wider, ko.Rmax_r, anorm,
                             bits_to_double(f->host_dev->xnorm_bits));
    }
    RUN(KC_STOREX, s, launch_store_x(n, f->TW, f->x, x, s));
    R.iters = k;
    R.status = (ir_solve_status)status;
    if (rep) {
        CK(cudaStreamSynchronize(s));
        *rep = R;
    }
    return IR_OK;
}

}  // namespace

extern "C" {

ir_status ir_solve_gmres(ir_fact *f, const void *b, void *x, const ir_term *term,
                         const ir_krylov_opts *kopts, void *stream, ir_report *rep, int *khist) {
    return krylov_solve(KRY_GMRES, f, b, x, term, kopts, stream, rep, khist);
}

ir_status ir_solve_bicgstab(ir_fact *f, const void *b, void *x, const ir_term *term,
                            const ir_krylov_opts *kopts, void *stream, ir_report *rep, int *khist) {
    return krylov_solve(KRY_BICGSTAB, f, b, x, term, kopts, stream, rep, khist);
}

namespace {

// The workspace of ir_solve_many's blocked path (allocated on first use).
ir_status ensure_multi(ir_fact *f) {
    if (f->xm) return IR_OK;
    const int64_t n = f->n;
    const int64_t nblk = (n + kTrsvB - 1) / kTrsvB;
    const size_t esz = (f->TW == IR_F64) ? 8 : 4;
    CK(cudaMalloc(&f->xm, (size_t)kMultiRhs * n * sizeof(double)));
    CK(cudaMalloc(&f->rm, (size_t)kMultiRhs * n * sizeof(double)));
    CK(cudaMalloc(&f->bm, (size_t)kMultiRhs * n * esz));
    CK(cudaMalloc(&f->mtags, (size_t)2 * kMultiRhs * nblk * kTrsvB * sizeof(unsigned long long)));
    CK(cudaMemset(f->mtags, 0, (size_t)2 * kMultiRhs * nblk * kTrsvB * sizeof(unsigned long long)));
    CK(cudaMalloc(&f->mscal, sizeof(MultiScalars)));
    CK(cudaMallocHost(&f->host_mscal, sizeof(MultiScalars)));
    return IR_OK;
}

// Several right-hand sides of one factorization refined together, up to 4 at a
// time: every correction solve applies each factor tile to all of the block's
// columns (launch_trsv_multi) and every residual reads A once for all of them
// (launch_residual_multi); each column keeps its own scaling (eq. vdlow), its
// own history and its own termination test (Sec. 5.1), and a column that has
// stopped takes no further corrections.
ir_status solve_many_blocked(ir_fact *f, int64_t nrhs, const void *B, int64_t ldb, void *X, int64_t ldx,
                             const ir_term &t, cudaStream_t s, ir_report *reps) {
    const int64_t n = f->n;
    const size_t esz = (f->TW == IR_F64) ? 8 : 4;
    ir_status st = ensure_multi(f);
    if (st != IR_OK) return st;
    // ns * n * 4 partial sums for the residual of 4 columns
    const int64_t need = residual_partials_needed(n, f->ctx->sms) * kMultiRhs;
    if (need > f->ctx->partials_cap) {
        if (f->ctx->partials) cudaFree(f->ctx->partials);
        f->ctx->partials = nullptr;
        f->ctx->partials_cap = 0;
        CK(cudaMalloc(&f->ctx->partials, need * sizeof(double)));
        f->ctx->partials_cap = need;
    }
    const bool tr_wider = (f->TW == IR_F32);
    const double eps_w = eps_of(f->TW);
    double anorm = 0.0;
    if (t.mode == 1) {
        if (!f->anorm_valid) RUN(KC_NORM1, s, launch_norm1(n, f->TW, f->A, f->lda, &f->dev->anorm_bits, s));
        st = read_dev(f, s);
        if (st != IR_OK) return st;
        f->anorm_valid = 1;
        anorm = bits_to_double(f->host_dev->anorm_bits);
    }
    ir_status first = IR_OK;
    MultiScalars *hm = f->host_mscal;
    for (int64_t c0 = 0; c0 < nrhs; c0 += kMultiRhs) {
        const int k = (int)((nrhs - c0 < kMultiRhs) ? nrhs - c0 : kMultiRhs);
        ir_report R[kMultiRhs];
        int status[kMultiRhs], iters[kMultiRhs];
        std::memset(R, 0, sizeof R);
        std::memset(hm, 0, sizeof(MultiScalars));
        // the block's right-hand sides (zero columns past k), x = 0, r = b, ||b||
        CK(cudaMemsetAsync(f->bm, 0, (size_t)kMultiRhs * n * esz, s));
        CK(cudaMemcpy2DAsync(f->bm, (size_t)n * esz, static_cast<const char *>(B) + (size_t)c0 * ldb * esz,
                             (size_t)ldb * esz, (size_t)n * esz, (size_t)k, cudaMemcpyDeviceToDevice, s));
        for (int j = 0; j < kMultiRhs; ++j) {
            R[j].scale = f->host_dev->scale;
            status[j] = IR_CONVERGED;
            iters[j] = 0;
            CK(cudaMemsetAsync(&f->dev->bnorm_bits, 0, sizeof(unsigned long long), s));
            CK(cudaMemsetAsync(&f->dev->nonfinite, 0, sizeof(int), s));
            RUN(KC_INIT, s, launch_init_rb(n, f->TW, static_cast<const char *>(f->bm) + (size_t)j * n * esz,
                                           f->rm + (size_t)j * n, f->xm + (size_t)j * n, f->dev, s));
            st = read_dev(f, s);
            if (st != IR_OK) return st;
            if (j >= k) continue;
            const double bn = bits_to_double(f->host_dev->bnorm_bits);
            R[j].rhist[0] = bn;
            hm->rho[j] = f->host_dev->bnorm_bits;
            if (f->host_dev->nonfinite) {
                status[j] = IR_FAILED;
                if (first == IR_OK) first = IR_ENONFINITE;
            } else if (bn != 0.0) {
                hm->active[j] = 1;
                status[j] = -1;
            }
        }
        CK(cudaMemcpyAsync(&f->mscal->rho, hm->rho, sizeof hm->rho, cudaMemcpyHostToDevice, s));
        int nactive = 0;
        for (int j = 0; j < kMultiRhs; ++j) nactive += hm->active[j];
        while (nactive > 0) {
            f->epoch += 1;
            CK(cudaMemcpyAsync(&f->mscal->active, hm->active, sizeof hm->active, cudaMemcpyHostToDevice, s));
            CK(cudaMemsetAsync(&f->mscal->dnorm, 0, sizeof hm->dnorm + sizeof hm->xnorm, s));
            RUN(KC_TRSV, s, launch_trsv_multi(f->AF, f->ldf, (int)n, f->Linv, f->Uinv, f->blk_subst, f->perm, f->rm,
                                              n, f->mscal->rho, f->mscal->active, f->xm, n, f->mscal->dnorm,
                                              f->mscal->xnorm, f->mtags, f->epoch, f->dev, s, f->AF16, f->TF));
            RUN(KC_RESID, s, launch_residual_multi(n, f->TW, f->A, f->lda, f->bm, n, f->xm, n, f->rm, n,
                                                   f->ctx->partials, f->ctx->partials_cap, f->mscal->rho,
                                                   f->ctx->sms, s));
            CK(cudaMemcpyAsync(hm, f->mscal, sizeof(MultiScalars), cudaMemcpyDeviceToHost, s));
            st = read_dev(f, s);     // synchronizes the stream (hm is current after it)
            if (st != IR_OK) return st;
            if (f->host_dev->timeout) {
                snprintf(g_last_error, sizeof g_last_error, "a bounded wait in the triangular solve timed out");
                return IR_ETIMEOUT;
            }
            for (int j = 0; j < k; ++j) {
                if (status[j] >= 0) continue;
                const int kk = ++iters[j];
                R[j].dhist[kk - 1] = bits_to_double(hm->dnorm[j]);
                R[j].rhist[kk] = bits_to_double(hm->rho[j]);
                const int d = term_decide(R[j].rhist, R[j].dhist, kk, R[j].rhist[0], eps_w, &t, tr_wider, t.Rmax,
                                          anorm, bits_to_double(hm->xnorm[j]));
                if (d >= 0) {
                    status[j] = d;
                    hm->active[j] = 0;
                    --nactive;
                }
            }
        }
        for (int j = 0; j < k; ++j) {
            if (status[j] != IR_FAILED)
                RUN(KC_STOREX, s, launch_store_x(n, f->TW, f->xm + (size_t)j * n,
                                                 static_cast<char *>(X) + (size_t)(c0 + j) * ldx * esz, s));
            R[j].iters = iters[j];
            R[j].status = (ir_solve_status)status[j];
            if (reps) reps[c0 + j] = R[j];
        }
    }
    CK(cudaMemsetAsync(&f->dev->nonfinite, 0, sizeof(int), s));   // a non-finite b is this call's, not the factorization's
    if (reps) CK(cudaStreamSynchronize(s));
    return first;
}

}  // namespace

ir_status ir_solve_many(ir_fact *f, int64_t nrhs, const void *B, int64_t ldb, void *X, int64_t ldx,
                        const ir_term *term, void *stream, ir_report *reps) {
    if (!f || nrhs < 0 || ldb < (f->n > 1 ? f->n : 1) || ldx < (f->n > 1 ? f->n : 1)) return IR_EINVAL;
    if (nrhs > 0 && f->n > 0 && (!B || !X)) return IR_EINVAL;
    ir_term t;
    if (term) t = *term;
    else ir_default_term(&t);
    if (t.litmax < 1 || t.litmax > IR_MAX_HIST - 1 || !(t.Rmax > 0) || (t.mode != 0 && t.mode != 1))
        return IR_EINVAL;
    const size_t esz = (f->TW == IR_F64) ? 8 : 4;
    cudaStream_t s = (cudaStream_t)stream;
    if (nrhs > 1 && f->n > 0 && !f->onthefly) {
        CK(cudaSetDevice(f->ctx->device));
        // the factorization's outcome, as ir_solve reports it
        ir_status st = read_dev(f, s);
        if (st != IR_OK) return st;
        const bool bad = f->host_dev->timeout || f->host_dev->nonfinite || f->host_dev->info != kInfoNone;
        if (!bad) return solve_many_blocked(f, nrhs, B, ldb, X, ldx, t, s, reps);
    }
    // one column at a time: a single right-hand side, mixed precision solves, or a
    // failed factorization (each ir_solve reports it)
    ir_status first = IR_OK;
    for (int64_t j = 0; j < nrhs; ++j) {
        const void *bj = static_cast<const char *>(B) + (size_t)j * ldb * esz;
        void *xj = static_cast<char *>(X) + (size_t)j * ldx * esz;
        const ir_status st = ir_solve(f, bj, xj, term, stream, reps ? reps + j : nullptr);
        if (st != IR_OK && first == IR_OK) first = st;
        if (st == IR_EINVAL || st == IR_ECUDA || st == IR_ENOMEM) return st;
    }
    return first;
}

ir_status ir_check_wait_timeout(ir_fact *f, double limit_s, void *stream) {
    if (!f || !(limit_s > 0.0) || limit_s * 1e9 > (double)kWaitLimitNs) return IR_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(f->ctx->device));
    CK(cudaMemsetAsync(&f->dev->timeout, 0, sizeof(int), s));
    // the tags carry solve epochs; epoch + 2^31 is never written by a solve
    const unsigned tag = f->epoch + 0x80000000u;
    CK(launch_wait_probe(f->tags, tag, (unsigned long long)(limit_s * 1e9), &f->dev->timeout, s));
    ir_status st = read_dev(f, s);
    if (st != IR_OK) return st;
    const int gave_up = f->host_dev->timeout;
    CK(cudaMemsetAsync(&f->dev->timeout, 0, sizeof(int), s));   // the factorization stays usable
    CK(cudaStreamSynchronize(s));
    if (gave_up) {
        snprintf(g_last_error, sizeof g_last_error, "the probe's bounded wait gave up after %.3g s", limit_s);
        return IR_ETIMEOUT;
    }
    return IR_OK;
}

ir_status ir_lu_solve(ir_fact *f, const float *v, float *d, void *stream) {
    if (!f || (f->n > 0 && (!v || !d))) return IR_EINVAL;
    if (f->n == 0) return IR_OK;
    CK(cudaSetDevice(f->ctx->device));
    f->epoch += 1;
    CK(launch_trsv_pair(f->AF, f->ldf, (int)f->n, f->Linv, f->Uinv, f->blk_subst, f->perm, nullptr, v, d, nullptr,
                        f->tags, f->epoch, f->dev, (cudaStream_t)stream, nullptr, nullptr, nullptr, false, f->AF16,
                        f->TF));
    return IR_OK;
}

ir_status ir_residual(ir_ctx *ctx, int64_t n, ir_dtype TW, const void *A, int64_t lda, const void *b,
                      const double *x, double *r, double *rnorm, void *stream) {
    if (!ctx || n < 0 || !tw_ok(TW) || lda < (n > 1 ? n : 1)) return IR_EINVAL;
    if (n > 0 && (!A || !b || !x || !r || !rnorm)) return IR_EINVAL;
    if (n == 0) {
        if (rnorm) CK(cudaMemsetAsync(rnorm, 0, sizeof(double), (cudaStream_t)stream));
        return IR_OK;
    }
    CK(cudaSetDevice(ctx->device));
    ir_status st = ensure_partials(ctx, n);
    if (st != IR_OK) return st;
    CK(launch_residual(n, TW, A, lda, b, x, r, ctx->partials, ctx->partials_cap,
                       reinterpret_cast<unsigned long long *>(rnorm), ctx->sms, (cudaStream_t)stream));
    return IR_OK;
}

ir_status ir_batch_create(ir_ctx *ctx, int64_t count, const int64_t *n_host, const void *const *A_dev,
                          const int64_t *lda_host, const void *const *b_dev, void *const *x_dev,
                          const ir_opts *opts, const ir_term *term, ir_batch **out) {
    if (!ctx || !out || count < 0) return IR_EINVAL;
    *out = nullptr;
    if (count > 0 && (!n_host || !A_dev || !b_dev || !x_dev)) return IR_EINVAL;
    if (count > INT_MAX / 2) return IR_EUNSUPPORTED;
    ir_opts o;
    if (opts) o = *opts;
    else ir_default_opts(&o);
    if (!tw_ok(o.TW) || !tf_ok(o.TF) || o.TR != IR_F64) return IR_EINVAL;
    if (o.nb != 0 && o.nb != kPanelNB) return IR_EUNSUPPORTED;
    ir_term t;
    if (term) t = *term;
    else ir_default_term(&t);
    if (t.litmax < 1 || t.litmax > IR_MAX_HIST - 1 || !(t.Rmax > 0) || (t.mode != 0 && t.mode != 1))
        return IR_EINVAL;
    if (t.mode != 0) return IR_EUNSUPPORTED;    // the batched driver tests small residuals (eq. residterm)
    int64_t maxn = 0;
    for (int64_t i = 0; i < count; ++i) {
        const int64_t n = n_host[i];
        const int64_t lda = lda_host ? lda_host[i] : (n > 1 ? n : 1);
        if (n < 0 || lda < (n > 1 ? n : 1)) return IR_EINVAL;
        if (n > 0 && (!A_dev[i] || !b_dev[i] || !x_dev[i])) return IR_EINVAL;
        if (n > IR_BATCH_MAX_N) {
            snprintf(g_last_error, sizeof g_last_error, "system %lld has n = %lld > IR_BATCH_MAX_N",
                     (long long)i, (long long)n);
            return IR_EUNSUPPORTED;
        }
        maxn = std::max(maxn, n);
    }
    CK(cudaSetDevice(ctx->device));
    ir_batch *b = new (std::nothrow) ir_batch();
    if (!b) return IR_ENOMEM;
    b->ctx = ctx;
    b->count = count;
    b->TW = o.TW;
    b->TF = o.TF;
    b->fp16_scale = o.fp16_scale;
    b->term = t;
    b->tc_min_trail = kPanelNB;
    ir_status st = IR_OK;
    cudaError_t e = batch_grid(ctx->sms, count, &b->grid);
    const int64_t cnt = count > 0 ? count : 1;
    // one slot per resident CTA: max n rows of (n rounded up to a multiple of 4) floats
    b->ws_stride = std::max<int64_t>((maxn * ((maxn + 3) / 4 * 4) + 31) / 32 * 32, 32);
    std::vector<unsigned char> desc(batch_desc_bytes() * cnt);
    std::vector<int> order(cnt, 0);
    for (int64_t i = 0; i < count; ++i) {
        const int64_t n = n_host[i];
        batch_fill_desc(desc.data(), i, A_dev[i], lda_host ? lda_host[i] : (n > 1 ? n : 1), b_dev[i], x_dev[i],
                        (int)n);
        order[i] = (int)i;
    }
    // longest first: the CTAs take the big systems first and the small ones fill the tail
    std::stable_sort(order.begin(), order.begin() + count,
                     [&](int x, int y) { return n_host[x] > n_host[y]; });
    if (e == cudaSuccess) e = cudaMalloc(&b->desc, desc.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->order, cnt * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->ticket, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&b->order2, cnt * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->count2, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&b->ws, (size_t)b->grid * b->ws_stride * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(b->desc, desc.data(), desc.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->order, order.data(), cnt * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        st = cuda_fail(e, "ir_batch_create");
        free_batch(b);
        return st;
    }
    if (o.autotune && count > 0 && (o.TF == IR_F16 || o.TF == IR_BF16)) {
        st = tune_batch(b);
        if (st != IR_OK) {
            free_batch(b);
            return st;
        }
    }
    *out = b;
    return IR_OK;
}

ir_status ir_batch_schedule(const ir_batch *b, int *grid, int *tc_min_trail) {
    if (!b) return IR_EINVAL;
    if (grid) *grid = b->grid;
    if (tc_min_trail) *tc_min_trail = b->tc_min_trail;
    return IR_OK;
}

ir_status ir_fact_schedule(const ir_fact *f, int *nb, int *panel_reserve_sms, int *group) {
    if (!f) return IR_EINVAL;
    if (nb) *nb = f->nb;
    if (panel_reserve_sms) *panel_reserve_sms = f->reserve_sms;
    if (group) *group = (f->TF != IR_F32 && f->Agrp) ? f->group : 1;
    return IR_OK;
}

ir_status ir_batch_run(ir_batch *b, ir_batch_result *results_dev, void *stream) {
    if (!b || (b->count > 0 && !results_dev)) return IR_EINVAL;
    if (b->count == 0) return IR_OK;
    CK(cudaSetDevice(b->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    RUN(KC_BATCHED, s, launch_batched(b->desc, b->order, b->count, b->ticket, b->ws, b->ws_stride, b->grid, b->TW,
                                      b->TF, b->fp16_scale, &b->term, b->tc_min_trail, results_dev, s));
    return IR_OK;
}

void ir_batch_destroy(ir_batch *b) { free_batch(b); }

ir_status ir_batch_run_escalate(ir_batch *b, ir_dtype tf2, double rtol, ir_batch_result *results_dev,
                                void *stream) {
    if (!b || (b->count > 0 && !results_dev) || (tf2 != IR_F32 && tf2 != IR_TF32) || !(rtol >= 0))
        return IR_EINVAL;
    ir_status st = ir_batch_run(b, results_dev, stream);
    if (st != IR_OK || b->count == 0) return st;
    cudaStream_t s = (cudaStream_t)stream;
    RUN(KC_BATCHED, s, launch_select_unconverged(results_dev, b->order, b->count, rtol, b->order2, b->count2, s));
    RUN(KC_BATCHED, s, launch_batched(b->desc, b->order2, b->count, b->ticket, b->ws, b->ws_stride, b->grid, b->TW,
                                      tf2, 0, &b->term, b->tc_min_trail, results_dev, s, b->count2));
    return IR_OK;
}

ir_status ir_factor_solve_batched(ir_ctx *ctx, int64_t count, const int64_t *n_host, const void *const *A_dev,
                                  const int64_t *lda_host, const void *const *b_dev, void *const *x_dev,
                                  const ir_opts *opts, const ir_term *term, void *stream,
                                  ir_batch_result *results_dev) {
    ir_batch *b = nullptr;
    ir_status st = ir_batch_create(ctx, count, n_host, A_dev, lda_host, b_dev, x_dev, opts, term, &b);
    if (st != IR_OK) return st;
    st = ir_batch_run(b, results_dev, stream);
    if (st == IR_OK) {
        const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) st = cuda_fail(e, "ir_factor_solve_batched");
    }
    ir_batch_destroy(b);
    return st;
}

ir_status ir_fact_pivots(const ir_fact *f, int32_t *ipiv_host) {
    if (!f || (f->n > 0 && !ipiv_host)) return IR_EINVAL;
    if (f->n == 0) return IR_OK;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(ipiv_host, f->ipiv, f->n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    return IR_OK;
}

ir_status ir_fact_factors(const ir_fact *f, float *LU_host, int64_t ld) {
    if (!f || ld < (f->n > 1 ? f->n : 1) || (f->n > 0 && !LU_host)) return IR_EINVAL;
    const int64_t n = f->n;
    if (n == 0) return IR_OK;
    float *tmp = (float *)std::malloc((size_t)n * f->ldf * sizeof(float));
    if (!tmp) return IR_ENOMEM;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(tmp, f->AF, (size_t)n * f->ldf * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        std::free(tmp);
        return cuda_fail(e, "ir_fact_factors");
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) LU_host[i + j * ld] = tmp[i * f->ldf + j];
    std::free(tmp);
    return IR_OK;
}

void ir_fact_destroy(ir_fact *f) { free_fact(f); }

ir_status ir_solve_host(ir_ctx *ctx, int64_t n, const void *A_host, int64_t lda, const void *b_host,
                        void *x_host, const ir_opts *opts, const ir_term *term, void *stream,
                        ir_report *rep) {
    if (!ctx || n < 0 || lda < (n > 1 ? n : 1)) return IR_EINVAL;
    if (n > 0 && (!A_host || !b_host || !x_host)) return IR_EINVAL;
    ir_opts o;
    if (opts) o = *opts;
    else ir_default_opts(&o);
    if (!tw_ok(o.TW)) return IR_EINVAL;
    const size_t es = o.TW == IR_F64 ? 8 : 4;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    const bool same = ctx->host_f && ctx->host_n == n && ctx->host_lda == lda && ctx->host_tw == (int)o.TW &&
                      ctx->host_tf == (int)o.TF && ctx->host_scale == o.fp16_scale &&
                      ctx->host_autotune == o.autotune && ctx->host_f->onthefly == o.onthefly &&
                      ctx->host_f->store_tf == o.store_tf &&
                      (o.group == 0 || ctx->host_f->group == o.group);
    if (!same) release_host_cache(ctx);
    ir_status st = IR_OK;
    cudaError_t e = cudaSuccess;
    const int64_t nn = n > 0 ? n : 1;
    if (!same) {
        e = cudaMalloc(&ctx->host_dA, (size_t)lda * nn * es);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->host_db, nn * es);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->host_dx, nn * es);
        if (e != cudaSuccess) {
            release_host_cache(ctx);
            return cuda_fail(e, "ir_solve_host allocation");
        }
    }
    if (n > 0) e = cudaMemcpyAsync(ctx->host_dA, A_host, (size_t)lda * n * es, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n > 0) e = cudaMemcpyAsync(ctx->host_db, b_host, n * es, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "ir_solve_host upload");
    if (same) {
        st = ir_refactor(ctx->host_f, ctx->host_dA, lda, stream);
    } else {
        st = ir_factor(ctx, n, ctx->host_dA, lda, &o, stream, &ctx->host_f);
        if (st == IR_OK) {
            ctx->host_n = n;
            ctx->host_lda = lda;
            ctx->host_tw = (int)o.TW;
            ctx->host_tf = (int)o.TF;
            ctx->host_scale = o.fp16_scale;
            ctx->host_autotune = o.autotune;
        }
    }
    if (st != IR_OK) {
        release_host_cache(ctx);
        return st;
    }
    st = ir_solve(ctx->host_f, ctx->host_db, ctx->host_dx, term, stream, rep);
    if (st != IR_OK) return st;
    if (n > 0) {
        e = cudaMemcpyAsync(x_host, ctx->host_dx, n * es, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "ir_solve_host download");
    }
    return st;
}

const char *ir_strerror(ir_status s) {
    switch (s) {
    case IR_OK: return "ok";
    case IR_EINVAL: return "invalid argument";
    case IR_ENOMEM: return "device allocation failed";
    case IR_ECUDA: return "CUDA runtime error";
    case IR_ESINGULAR: return "zero pivot in the factorization";
    case IR_ENONFINITE: return "non-finite value in A, b or the rounded copy";
    case IR_ETIMEOUT: return "a bounded device wait timed out";
    case IR_EUNSUPPORTED: return "unsupported size or configuration";
    }
    return "unknown status";
}

}  // extern "C"
