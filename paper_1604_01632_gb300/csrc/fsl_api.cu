// fsl_api.cu -- the C ABI of include/fsl.h: device memory, stream ordering,
// step graphs, state exports.  Host code only; kernels live in fsl_core.cu
// (precision-independent + FP64) and fsl_fast.cu (FP32 / FP16 / BF16 forms).
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <string>
#include <vector>

#include "../../include/fsl.h"
#include "fsl_device.cuh"
#include "fsl_internal.h"

using namespace fsl;

namespace {

const int kDefaultCapacityMin = 256;

// Candidate sequence of the autotuner: every form twice, the faster of its two
// timed steps counts (the slab form only where the interface list is kept in
// cell order; it is skipped otherwise).
const int kTuneSeq[] = {SC_SPLIT, SC_PERS1, SC_PERS2, SC_PERS4, SC_SLAB, SC_TWO, SC_TILE2, SC_TILE4, SC_TWOC,
                        SC_SPLIT, SC_PERS1, SC_PERS2, SC_PERS4, SC_SLAB, SC_TWO, SC_TILE2, SC_TILE4, SC_TWOC};
const int kTuneSteps = (int)(sizeof(kTuneSeq) / sizeof(kTuneSeq[0]));

// Process-wide cache of tuning decisions, keyed by the workload's shape:
// storage precision, one or many domains, SM count, lattice size (log2 of the
// padded cells) and the interface share (in 1/64 steps) at tuning time.
struct TuneKey {
    int prec, multi, sms, lsize, ifrac;
    bool operator<(const TuneKey& o) const {
        if (prec != o.prec) return prec < o.prec;
        if (multi != o.multi) return multi < o.multi;
        if (sms != o.sms) return sms < o.sms;
        if (lsize != o.lsize) return lsize < o.lsize;
        return ifrac < o.ifrac;
    }
};
std::mutex g_tune_mutex;
std::map<TuneKey, int> g_tune_cache;

}  // namespace

struct fsl_domain {
    int ndom = 0;
    int precision = 0;
    size_t fbytes = 8;            // bytes per stored PDF
    cudaStream_t user = nullptr;  // caller's stream (may be the legacy default)
    cudaStream_t ls = nullptr;    // library stream (capturable)
    cudaStream_t ls2 = nullptr;   // second stream of the two-stream stream-collide form
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    int ifblocks = 304;           // grid of the list kernels (2 blocks per SM)
    int form = SC_SPLIT;          // stream-collide kernel form in use
    // autotuner: while `tuning`, each step runs the next candidate form with
    // CUDA events around its stream-collide kernel (direct launches)
    bool tuning = true;           // auto mode and not yet decided
    int tune_next = 0;            // index into the candidate sequence
    double tune_ms[SC_FORMS] = {};   // best measured time per form (0: not run)
    int tune_source = 0;          // 0 none yet, 1 measured here, 2 taken from the process cache, 3 fixed by the caller
    cudaEvent_t tev[2] = {nullptr, nullptr};
    int order_mode = -1;          // interface list in cell order: 1 on, 0 off, -1 by lattice size
    long long l2bytes = 0;        // L2 cache of the device
    int* ocnt = nullptr;          // interface cells per conversion block (ordered rebuild)
    int pgrid[SC_FORMS] = {};     // resident grid of each persistent form
    int convblocks = 152;         // grid of the cooperative conversion kernel
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<fsl_params> params;
    std::vector<Dom> hdoms;
    long long stride = 0;          // padded cells
    long long nblocks = 0;
    long long nslots = 0;
    std::vector<int> blk_dom;
    std::vector<int> slot_dom;

    // device state
    Dom* d_doms = nullptr;
    int* d_blk_dom = nullptr;
    int4* d_ntiles = nullptr;      // normals-pass tiles of a batch (null: some domain is smaller)
    int nntiles = 0;
    int* d_slot_dom = nullptr;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    uint8_t *flag = nullptr, *mark = nullptr;
    double *m = nullptr, *phi = nullptr, *phit = nullptr, *rhoi = nullptr, *exs = nullptr;
    float *phif = nullptr, *phitf = nullptr;   // FP32 copies (FP32-collide forms only)
    void* nrm = nullptr;           // normals pass: 3 planes of the arithmetic type
    unsigned* nmask = nullptr;     // normals pass: reconstruction directions per interface cell
    void* pvc = nullptr;           // normals pass: bubble pressure per interface cell
    int* id = nullptr;
    long long *vfx = nullptr, *vxfx = nullptr, *vsfx = nullptr, *ncells = nullptr;
    int* constp = nullptr;
    long long *pool = nullptr, *nif = nullptr;
    int* trig = nullptr;
    int* status = nullptr;
    unsigned* bar = nullptr;      // grid barrier of the conversion kernel
    int* ilist[2] = {nullptr, nullptr};   // interface list read by a step starting from buffer k
    int* icount[2] = {nullptr, nullptr};
    int *mlist = nullptr, *mcount = nullptr, *glist = nullptr, *gcount = nullptr, *llist = nullptr, *lcount = nullptr;
    int *cstep = nullptr, *recv = nullptr, *stepno = nullptr;
    long long* icnt = nullptr;
    // labelling scratch
    int *lab = nullptr, *aux = nullptr;
    unsigned long long* hkeys = nullptr;
    long long* hvals = nullptr;
    long long hcap = 0;
    long long *nvfx = nullptr, *nvxfx = nullptr, *nvsfx = nullptr, *nncells = nullptr;
    int *nconstp = nullptr, *croot = nullptr, *minc = nullptr;
    int *hused = nullptr, *nhused = nullptr, *nused = nullptr, *nfree = nullptr, *freelist = nullptr;
    int *aff = nullptr, *afflist = nullptr, *naff = nullptr, *plist = nullptr, *np = nullptr;
    int *newslots = nullptr, *nnew = nullptr;
    int* bbox = nullptr;                 // per slot: box of its cells (6 ints)
    long long *rowoff = nullptr, *nrows = nullptr;   // box rows of the marked slots
    long long* vtot = nullptr;
    int* minidx = nullptr;
    long long* counts = nullptr;
    double* mass_part = nullptr;  // per-block liquid-mass sums (fsl_total_mass)
    long long max_dom_blocks = 1;
    long long* runs = nullptr;

    std::vector<bool> inited;
    bool need_initial_ccl = true;
    bool stepped = false;
    // step graphs: [starting buffer][kind]; kind 0 = two steps, 1 = one step,
    // 2 = one step with event-record nodes around the stream-collide kernels
    cudaGraphExec_t graph[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    cudaGraphNode_t rec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    cudaGraph_t timed_src[2] = {nullptr, nullptr};   // kept: its nodes name the event records
    int graph_kernels[3] = {0, 0, 0};
    long long launches = 0;
    int ccl_cap = 1 << 24;        // cap on the labelling's union / find loops
    int spins = 1 << 22;          // polls at a grid barrier before FSL_ERR_SYNC
    int bar_extra = 0;            // 1: barriers wait for a block that does not exist (tests)
    bool timing = false;
    bool graphs = true;           // false: every kernel a separate launch (profilers)
    std::vector<cudaEvent_t> evpool;
    size_t evused = 0;
    double k1_ms = 0.0;
    std::vector<cudaEvent_t> phpool;   // direct mode: events between the kernels of a step
    size_t phused = 0;
    double phase_ms[4] = {0, 0, 0, 0};
    std::vector<void*> allocs;
    void* stage = nullptr;        // device staging of host transfers (init, export), grown on demand
    size_t stage_bytes = 0;
    std::string err;
};

namespace {

fsl_status fail(fsl_domain* h, fsl_status st, const std::string& msg) {
    if (h) h->err = msg;
    return st;
}

fsl_status cuda_fail(fsl_domain* h, cudaError_t e, const char* where) {
    return fail(h, FSL_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                              \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
    } while (0)

template <typename P>
cudaError_t dalloc(fsl_domain* h, P** p, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes > 0 ? bytes : 16);
    if (e == cudaSuccess) {
        h->allocs.push_back(q);
        *p = (P*)q;
    }
    return e;
}

// Device staging for transfers from or to host buffers: one buffer owned by
// the handle, grown when a call needs more (freeing the old one waits for the
// device), so that repeated calls neither allocate nor synchronise the device
// for an allocation.  parts[i] receives a 256-byte aligned slice of bytes[i].
cudaError_t staging(fsl_domain* h, const size_t* bytes, int n, void** parts) {
    size_t tot = 0;
    for (int i = 0; i < n; ++i) tot += (bytes[i] + 255) / 256 * 256;
    if (tot > h->stage_bytes) {
        if (h->stage) cudaFree(h->stage);
        h->stage = nullptr;
        h->stage_bytes = 0;
        cudaError_t e = cudaMalloc(&h->stage, tot);
        if (e != cudaSuccess) return e;
        h->stage_bytes = tot;
    }
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        parts[i] = (char*)h->stage + off;
        off += (bytes[i] + 255) / 256 * 256;
    }
    return cudaSuccess;
}

// Whether the conversion kernel rebuilds the interface list in cell order: by
// default where the two PDF arrays of a step exceed twice the L2 cache (there
// an interface cell's neighbour data would otherwise come from DRAM again for
// every cell that reads it; the rebuild reads the cell types twice).
// Kernels one step launches with stream-collide form f: the conversion kernel,
// plus the normals pass in the forms that take interface cells one per thread,
// plus one or two stream-collide kernels.
int kernels_per_step(int f) {
    if (f == SC_TWO || f == SC_TWOC) return 4;
    if (f == SC_TILE2 || f == SC_TILE4) return 3;
    return 2;
}

int order_effective(const fsl_domain* h) {
    if (h->order_mode >= 0) return h->order_mode;
    const double pdf_bytes = 2.0 * 19.0 * (double)h->stride * (double)h->fbytes;
    return h->l2bytes > 0 && pdf_bytes > 2.0 * (double)h->l2bytes ? 1 : 0;
}

StepArgs step_args(fsl_domain* h, int src) {
    StepArgs A;
    A.doms = h->d_doms;
    A.blk_dom = h->d_blk_dom;
    A.ntiles = h->d_ntiles;
    A.nntiles = h->nntiles;
    A.stride = h->stride;
    A.fsrc = h->f[src];
    A.fdst = h->f[1 - src];
    A.flag = h->flag;
    A.mark = h->mark;
    A.m = h->m;
    A.phi = h->phi;
    A.phit = h->phit;
    A.phif = h->phif;
    A.phitf = h->phitf;
    A.bbox = h->bbox;
    A.nrm = h->nrm;
    A.nmask = h->nmask;
    A.pvc = h->pvc;
    A.rhoi = h->rhoi;
    A.exs = h->exs;
    A.id = h->id;
    A.vfx = h->vfx;
    A.vxfx = h->vxfx;
    A.vsfx = h->vsfx;
    A.ncells = h->ncells;
    A.constp = h->constp;
    A.pool = h->pool;
    A.nif = h->nif;
    A.trig = h->trig;
    A.status = h->status;
    A.bar = h->bar;
    A.order = order_effective(h);
    A.ocnt = h->ocnt;
    A.spins = h->spins;
    A.bar_extra = h->bar_extra;
    A.ndom = h->ndom;
    A.ilist = h->ilist[src];
    A.icount = h->icount[src];
    A.ilist_next = h->ilist[1 - src];
    A.icount_next = h->icount[1 - src];
    A.mlist = h->mlist;
    A.mcount = h->mcount;
    A.glist = h->glist;
    A.gcount = h->gcount;
    A.llist = h->llist;
    A.lcount = h->lcount;
    A.cstep = h->cstep;
    A.recv = h->recv;
    A.stepno = h->stepno;
    A.icnt = h->icnt;
    A.d0 = h->hdoms[0];
    return A;
}

CclArgs ccl_args(fsl_domain* h, int initial) {
    CclArgs K;
    K.lab = h->lab;
    K.aux = h->aux;
    K.hkeys = h->hkeys;
    K.hvals = h->hvals;
    K.hcap = h->hcap;
    K.nvfx = h->nvfx;
    K.nvxfx = h->nvxfx;
    K.nvsfx = h->nvsfx;
    K.nncells = h->nncells;
    K.nconstp = h->nconstp;
    K.croot = h->croot;
    K.vtot = h->vtot;
    K.minc = h->minc;
    K.hused = h->hused;
    K.nhused = h->nhused;
    K.nused = h->nused;
    K.nfree = h->nfree;
    K.freelist = h->freelist;
    K.aff = h->aff;
    K.afflist = h->afflist;
    K.naff = h->naff;
    K.plist = h->plist;
    K.np = h->np;
    K.newslots = h->newslots;
    K.nnew = h->nnew;
    K.rowoff = h->rowoff;
    K.nrows = h->nrows;
    K.slot_dom = h->d_slot_dom;
    K.runs = h->runs;
    K.vsfx = h->vsfx;
    K.constp = h->constp;
    K.initial = initial;
    // find() walks strictly decreasing indices and every retry of unite()
    // follows a link made by another thread, so both loops end; the caps only
    // turn a corrupted label array into an error status
    K.max_iter = h->ccl_cap;
    return K;
}

void launch_k1(fsl_domain* h, const StepArgs& A, cudaStream_t st, cudaEvent_t el = nullptr, cudaEvent_t ei = nullptr,
               int form = -1) {
    if (form < 0) form = h->form;
    const int pg = h->pgrid[form];
    cudaStream_t s2 = h->ls2;
    cudaEvent_t fk = h->ev_fork, jn = h->ev_join;
    switch (h->precision) {
    case FSL_P_FP64: launch_stream<double>(A, h->nblocks, h->ifblocks, form, pg, st, el, ei, s2, fk, jn); break;
    case FSL_P_FP32: launch_stream<float>(A, h->nblocks, h->ifblocks, form, pg, st, el, ei, s2, fk, jn); break;
    case FSL_P_F16S: launch_stream<__half>(A, h->nblocks, h->ifblocks, form, pg, st, el, ei, s2, fk, jn); break;
    default: launch_stream<__nv_bfloat16>(A, h->nblocks, h->ifblocks, form, pg, st, el, ei, s2, fk, jn); break;
    }
}

int stream_occupancy(int precision, int form, bool one) {
    switch (precision) {
    case FSL_P_FP64: return stream_blocks_per_sm<double>(form, one);
    case FSL_P_FP32: return stream_blocks_per_sm<float>(form, one);
    case FSL_P_F16S: return stream_blocks_per_sm<__half>(form, one);
    default: return stream_blocks_per_sm<__nv_bfloat16>(form, one);
    }
}

// form: the stream-collide form the conversion kernel follows (after the
// two-stream form it depends on a join, not programmatically on one kernel)
cudaError_t launch_conv(fsl_domain* h, const StepArgs& A, cudaStream_t st, int form = -1) {
    const CclArgs K = ccl_args(h, 0);
    const bool pdl = (form < 0 ? h->form : form) != SC_TWOC;
    switch (h->precision) {
    case FSL_P_FP64: return launch_convert<double>(A, K, h->convblocks, st, pdl);
    case FSL_P_FP32: return launch_convert<float>(A, K, h->convblocks, st, pdl);
    case FSL_P_F16S: return launch_convert<__half>(A, K, h->convblocks, st, pdl);
    default: return launch_convert<__nv_bfloat16>(A, K, h->convblocks, st, pdl);
    }
}

int conv_blocks_per_sm(int precision) {
    switch (precision) {
    case FSL_P_FP64: return convert_blocks_per_sm<double>();
    case FSL_P_FP32: return convert_blocks_per_sm<float>();
    case FSL_P_F16S: return convert_blocks_per_sm<__half>();
    default: return convert_blocks_per_sm<__nv_bfloat16>();
    }
}

// The stream-collide kernel and the conversion kernel of one step (2
// kernels).  With e0/e1 the stream-collide kernel is bracketed by event
// records (captured as event-record nodes when the stream is capturing; their
// nodes go to rec).
cudaEvent_t next_phase_event(fsl_domain* h) {
    while (h->phpool.size() < h->phused + 1) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        h->phpool.push_back(e);
    }
    return h->phpool[h->phused++];
}

int enqueue_main(fsl_domain* h, const StepArgs& A, cudaEvent_t e0, cudaEvent_t e1, cudaGraphNode_t* rec,
                 bool phases = false) {
    auto last_node = [&](int k) {
        if (!rec) return;
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        if (cudaStreamGetCaptureInfo(h->ls, &cs, nullptr, nullptr, &deps, nullptr, &nd) == cudaSuccess && nd == 1)
            rec[k] = deps[0];
    };
    // while capturing (rec given) the records are external, so that the
    // capture turns them into event-record nodes
    auto record = [&](cudaEvent_t e) {
        if (rec) cudaEventRecordWithFlags(e, h->ls, cudaEventRecordExternal);
        else cudaEventRecord(e, h->ls);
    };
    if (e0) { record(e0); last_node(0); }
    if (phases) {
        cudaEvent_t el = next_phase_event(h), ei = next_phase_event(h);
        launch_k1(h, A, h->ls, el, ei);
    } else {
        launch_k1(h, A, h->ls);
    }
    if (e1) { record(e1); last_node(1); }
    launch_conv(h, A, h->ls);
    if (phases) cudaEventRecord(next_phase_event(h), h->ls);
    return kernels_per_step(h->form);
}

std::pair<cudaEvent_t, cudaEvent_t> next_events(fsl_domain* h) {
    while (h->evpool.size() < h->evused + 2) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        h->evpool.push_back(e);
    }
    cudaEvent_t a = h->evpool[h->evused++];
    cudaEvent_t b = h->evpool[h->evused++];
    return {a, b};
}

// Order library work after the caller's stream, and the caller after it.
void join_in(fsl_domain* h) {
    cudaEventRecord(h->ev_in, h->user);
    cudaStreamWaitEvent(h->ls, h->ev_in, 0);
}
void join_out(fsl_domain* h) {
    cudaEventRecord(h->ev_out, h->ls);
    cudaStreamWaitEvent(h->user, h->ev_out, 0);
}

fsl_status latch(fsl_domain* h) {
    int st = 0;
    cudaError_t e = cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "status read");
    if (st != 0) {
        const char* what = st == FSL_ERR_GEOMETRY ? "a liquid cell touches a gas cell"
                           : st == FSL_ERR_NAN ? "a density became NaN"
                           : st == FSL_ERR_CCL_NOT_CONVERGED ? "bubble labelling hit its iteration cap"
                           : st == FSL_ERR_TABLE_FULL ? "bubble table full"
                           : st == FSL_ERR_SYNC ? "a grid barrier of the conversion kernel timed out"
                                                : "device error";
        // a barrier that timed out leaves its arrival count behind
        if (st == FSL_ERR_SYNC) cudaMemset(h->bar, 0, 2 * sizeof(unsigned));
        return fail(h, (fsl_status)st, what);
    }
    return FSL_OK;
}

fsl_status ensure_initial(fsl_domain* h) {
    if (!h->need_initial_ccl) return FSL_OK;
    for (int d = 0; d < h->ndom; ++d)
        if (!h->inited[d]) return fail(h, FSL_ERR_ARG, "every domain must be initialised first");
    StepArgs A = step_args(h, h->cur);
    // the initial pass hands out every slot afresh and rebuilds every table row
    const size_t NS = (size_t)h->nslots;
    CK(h, cudaMemsetAsync(h->nused, 0, 4 * (size_t)h->ndom, h->ls));
    CK(h, cudaMemsetAsync(h->nfree, 0, 4 * (size_t)h->ndom, h->ls));
    CK(h, cudaMemsetAsync(h->aff, 0, 4 * NS, h->ls));
    CK(h, cudaMemsetAsync(h->naff, 0, sizeof(int), h->ls));
    CK(h, cudaMemsetAsync(h->np, 0, sizeof(int), h->ls));
    CK(h, cudaMemsetAsync(h->nnew, 0, sizeof(int), h->ls));
    CK(h, cudaMemsetAsync(h->nhused, 0, sizeof(int), h->ls));
    CK(h, cudaMemsetAsync(h->vfx, 0, 8 * NS, h->ls));
    CK(h, cudaMemsetAsync(h->vxfx, 0, 8 * NS, h->ls));
    CK(h, cudaMemsetAsync(h->vsfx, 0, 8 * NS, h->ls));
    CK(h, cudaMemsetAsync(h->ncells, 0, 8 * NS, h->ls));
    CK(h, cudaMemsetAsync(h->constp, 0, 4 * NS, h->ls));
    h->launches += launch_ccl(A, ccl_args(h, 1), h->nblocks, h->ls);
    CK(h, cudaMemsetAsync(h->icount[h->cur], 0, sizeof(int), h->ls));
    CK(h, cudaMemsetAsync(h->icnt, 0, 8 * (size_t)h->ndom, h->ls));
    launch_build_ilist(A, h->nblocks, h->ls);
    h->launches += 1;
    CK(h, cudaGetLastError());
    h->need_initial_ccl = false;
    return FSL_OK;
}

// One or two steps starting from buffer `start` as one graph (per step: the
// stream-collide kernel, then the cooperative conversion kernel, which also
// runs the labelling on trigger steps).  kind 2 brackets the stream-collide
// kernel with event-record nodes whose events are swapped before every
// launch.
fsl_status build_graph(fsl_domain* h, int start, int kind) {
    const int nsteps = kind == 0 ? 2 : 1;
    cudaGraph_t G = nullptr;
    CK(h, cudaGraphCreate(&G, 0));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (kind == 2) {
        auto ev = next_events(h);
        e0 = ev.first;
        e1 = ev.second;
    }
    CK(h, cudaStreamBeginCaptureToGraph(h->ls, G, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    int kk = 0;
    for (int j = 0; j < nsteps; ++j) {
        StepArgs A = step_args(h, j == 0 ? start : 1 - start);
        kk += enqueue_main(h, A, e0, e1, kind == 2 ? h->rec[start] : nullptr);
    }
    cudaGraph_t out = nullptr;
    CK(h, cudaStreamEndCapture(h->ls, &out));
    if (kind == 2 && (!h->rec[start][0] || !h->rec[start][1])) {
        cudaGraphDestroy(G);
        return fail(h, FSL_ERR_CUDA, "event-record nodes not found in the captured step");
    }
    CK(h, cudaGraphInstantiate(&h->graph[start][kind], G, 0));
    if (kind == 2) h->timed_src[start] = G;
    else cudaGraphDestroy(G);
    h->graph_kernels[kind] = kk;
    if (kind == 2) h->evused -= 2;  // the capture events are placeholders
    return FSL_OK;
}

fsl_status launch_graph(fsl_domain* h, int kind) {
    if (!h->graph[h->cur][kind]) {
        fsl_status gs = build_graph(h, h->cur, kind);
        if (gs != FSL_OK) return gs;
    }
    if (kind == 2) {
        auto ev = next_events(h);
        CK(h, cudaGraphExecEventRecordNodeSetEvent(h->graph[h->cur][2], h->rec[h->cur][0], ev.first));
        CK(h, cudaGraphExecEventRecordNodeSetEvent(h->graph[h->cur][2], h->rec[h->cur][1], ev.second));
    }
    CK(h, cudaGraphLaunch(h->graph[h->cur][kind], h->ls));
    h->launches += h->graph_kernels[kind];
    return FSL_OK;
}

}  // namespace

extern "C" {

fsl_status fsl_create(const fsl_params* params, int32_t n_domains, int32_t precision, void* cuda_stream,
                      fsl_domain** out) {
    if (!params || !out || n_domains <= 0 || precision < 0 || precision > 3) return FSL_ERR_ARG;
    *out = nullptr;
    fsl_domain* h = new fsl_domain();
    h->ndom = n_domains;
    h->precision = precision;
    h->fbytes = precision == FSL_P_FP64 ? 8 : (precision == FSL_P_FP32 ? 4 : 2);
    h->user = (cudaStream_t)cuda_stream;
    long long off = 0;
    long long soff = 0;
    for (int d = 0; d < n_domains; ++d) {
        const fsl_params& p = params[d];
        long long n = (long long)p.nx * p.ny * p.nz;
        if (p.nx <= 0 || p.ny <= 0 || p.nz <= 0 || n >= (1LL << 31) || !(p.tau > 0.5) || p.split_trigger < 0 ||
            p.split_trigger > 1) {
            delete h;
            return FSL_ERR_ARG;
        }
        h->params.push_back(p);
        Dom D;
        memset(&D, 0, sizeof(D));
        D.nx = p.nx; D.ny = p.ny; D.nz = p.nz; D.n = (int)n;
        D.off = off;
        long long cap = p.bubble_capacity > 0 ? p.bubble_capacity : std::max<long long>(kDefaultCapacityMin, n / 64);
        D.slot_off = (int)soff;
        D.slot_cap = (int)cap;
        D.seed = -1;
        D.normal_rule = p.normal_rule;
        D.rate_fx = 0;
        D.omp = 1.0 / p.tau;
        D.omm = p.collision == FSL_TRT ? 1.0 / (p.magic / (p.tau - 0.5) + 0.5) : D.omp;
        D.sigma2 = 2.0 * p.sigma;
        for (int k = 0; k < 3; ++k) { D.g[k] = p.gravity[k]; D.lid[k] = p.lid_velocity[k]; }
        D.eps = p.eps;
        D.fomp = (float)D.omp;
        D.fomm = (float)D.omm;
        D.fsigma2 = (float)D.sigma2;
        for (int k = 0; k < 3; ++k) { D.fg[k] = (float)D.g[k]; D.flid[k] = (float)D.lid[k]; }
        D.feps = (float)D.eps;
        div_magic(p.nx, D.mgx, D.shx);
        div_magic(p.ny, D.mgy, D.shy);
        D.has_force = (p.gravity[0] != 0.0 || p.gravity[1] != 0.0 || p.gravity[2] != 0.0) ? 1 : 0;
        D.lonely_rule = p.lonely_rule;
        D.split_trigger = p.split_trigger;
        h->hdoms.push_back(D);
        long long padded = (n + FSL_BLOCK - 1) / FSL_BLOCK * FSL_BLOCK;
        for (long long b = 0; b < padded / FSL_BLOCK; ++b) h->blk_dom.push_back(d);
        for (long long s = 0; s < cap; ++s) h->slot_dom.push_back(d);
        off += padded;
        soff += cap;
    }
    // cell numbers are 31-bit and the kernels address PDFs with 32-bit offsets
    if (off >= (1LL << 31) || 19 * off >= (1LL << 32) || soff >= (1LL << 31)) { delete h; return FSL_ERR_ARG; }
    h->stride = off;
    h->nblocks = off / FSL_BLOCK;
    h->nslots = soff;
    h->inited.assign(n_domains, false);
    long long hc = 1024;
    while (hc < 4 * soff) hc <<= 1;
    h->hcap = hc;

    cudaError_t e = cudaStreamCreateWithFlags(&h->ls, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms > 0) h->ifblocks = 2 * sms;
        // the cooperative conversion kernel: all blocks resident; as many as
        // fit, because on trigger steps its labelling phases sweep the whole
        // lattice (a barrier over more blocks costs a little more)
        const int per_sm = conv_blocks_per_sm(precision);
        if (per_sm < 1) e = cudaErrorInvalidConfiguration;
        h->convblocks = std::max(1, sms) * std::max(1, per_sm);
        int l2 = 0;
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
        h->l2bytes = l2;
        for (int f = SC_PERS1; f < SC_FORMS; ++f)
            h->pgrid[f] = std::max(1, sms) * std::max(1, stream_occupancy(precision, f, n_domains == 1));
        // beside the liquid kernel the interface kernel keeps half its blocks per SM
        h->pgrid[SC_TWOC] = std::max(1, sms) * std::max(1, stream_occupancy(precision, SC_TWOC, n_domains == 1) / 2);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->ls2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
    const size_t N = (size_t)h->stride, NS = (size_t)h->nslots;
#define AL(ptr, bytes) if (e == cudaSuccess) e = dalloc(h, &(ptr), (bytes))
    AL(h->d_doms, sizeof(Dom) * n_domains);
    AL(h->d_blk_dom, sizeof(int) * h->blk_dom.size());
    // tiles of the normals pass over a batch, when every domain holds a whole tile
    std::vector<int4> ntl;
    bool tiled = n_domains > 1;
    for (const Dom& D : h->hdoms) tiled = tiled && D.nx >= NT_X && D.ny >= NT_Y && D.nz >= NT_Z;
    if (tiled) {
        for (int d = 0; d < n_domains; ++d) {
            const Dom& D = h->hdoms[d];
            for (int z0 = 0; z0 < D.nz; z0 += NT_Z)
                for (int y0 = 0; y0 < D.ny; y0 += NT_Y)
                    for (int x0 = 0; x0 < D.nx; x0 += NT_X) ntl.push_back(make_int4(d, x0, y0, z0));
        }
        h->nntiles = (int)ntl.size();
        AL(h->d_ntiles, sizeof(int4) * ntl.size());
    }
    AL(h->d_slot_dom, sizeof(int) * NS);
    AL(h->f[0], 19 * N * h->fbytes);
    AL(h->f[1], 19 * N * h->fbytes);
    AL(h->flag, N);
    AL(h->mark, N);
    AL(h->m, 8 * N);
    AL(h->phi, 8 * N);
    AL(h->phit, 8 * N);
    if (precision != FSL_P_FP64) {
        AL(h->phif, 4 * N);
        AL(h->phitf, 4 * N);
    }
    AL(h->nrm, 3 * N * (precision == FSL_P_FP64 ? 8 : 4));
    AL(h->nmask, 4 * N);
    AL(h->pvc, N * (precision == FSL_P_FP64 ? 8 : 4));
    AL(h->rhoi, 8 * N);
    AL(h->exs, 8 * N);
    AL(h->id, 4 * N);
    AL(h->vfx, 8 * NS);
    AL(h->vxfx, 8 * NS);
    AL(h->vsfx, 8 * NS);
    AL(h->ncells, 8 * NS);
    AL(h->constp, 4 * NS);
    AL(h->pool, 8 * n_domains);
    AL(h->nif, 8 * n_domains);
    AL(h->trig, sizeof(int) * (n_domains + 1));
    AL(h->status, sizeof(int));
    AL(h->bar, 2 * sizeof(unsigned));
    AL(h->ilist[0], 4 * N);
    AL(h->ilist[1], 4 * N);
    AL(h->icount[0], sizeof(int));
    AL(h->icount[1], sizeof(int));
    AL(h->mlist, 4 * N);
    AL(h->mcount, sizeof(int));
    AL(h->glist, 4 * N);
    AL(h->gcount, sizeof(int));
    AL(h->llist, 4 * N);
    AL(h->lcount, sizeof(int));
    AL(h->cstep, 4 * N);
    AL(h->recv, 4 * N);
    AL(h->stepno, sizeof(int));
    AL(h->icnt, 8 * n_domains);

    AL(h->lab, 4 * N);
    AL(h->aux, 4 * N);
    AL(h->hkeys, 8 * (size_t)hc);
    AL(h->hvals, 8 * (size_t)hc);
    AL(h->nvfx, 8 * NS);
    AL(h->nvxfx, 8 * NS);
    AL(h->nvsfx, 8 * NS);
    AL(h->nncells, 8 * NS);
    AL(h->nconstp, 4 * NS);
    AL(h->croot, 4 * NS);
    AL(h->minc, 4 * NS);
    AL(h->vtot, 8 * NS);
    AL(h->ocnt, 4 * (size_t)h->convblocks);
    AL(h->hused, 4 * (size_t)hc);
    AL(h->nhused, sizeof(int));
    AL(h->nused, 4 * n_domains);
    AL(h->nfree, 4 * n_domains);
    AL(h->freelist, 4 * NS);
    AL(h->aff, 4 * NS);
    AL(h->afflist, 4 * NS);
    AL(h->naff, sizeof(int));
    AL(h->plist, 4 * N);
    AL(h->np, sizeof(int));
    AL(h->newslots, 4 * NS);
    AL(h->nnew, sizeof(int));
    AL(h->bbox, 6 * 4 * NS);
    AL(h->rowoff, 8 * NS);
    AL(h->nrows, 8);
    AL(h->minidx, 4 * NS);
    AL(h->counts, 8 * 8);
    for (const Dom& D : h->hdoms) h->max_dom_blocks = std::max(h->max_dom_blocks, ((long long)D.n + FSL_BLOCK - 1) / FSL_BLOCK);
    AL(h->mass_part, 8 * (size_t)h->max_dom_blocks);
    AL(h->runs, 16);   // [0] labelling passes, [1] bubbles they relabelled
#undef AL
    // the staging buffer of fsl_init_geometry from host buffers, sized for the
    // largest domain, taken now with every other buffer rather than inside the
    // first upload (it grows later only for larger exports)
    if (e == cudaSuccess) {
        long long nmax = 0;
        for (const Dom& D : h->hdoms) nmax = std::max(nmax, (long long)D.n);
        const size_t bytes[4] = {(size_t)nmax, 8 * (size_t)nmax, 8 * (size_t)nmax, 24 * (size_t)nmax};
        void* parts[4];
        e = staging(h, bytes, 4, parts);
    }
    if (e != cudaSuccess) {
        fsl_status st = (e == cudaErrorMemoryAllocation) ? FSL_ERR_OOM : FSL_ERR_CUDA;
        fsl_destroy(h);
        return st;
    }
    e = cudaMemcpy(h->d_doms, h->hdoms.data(), sizeof(Dom) * n_domains, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_blk_dom, h->blk_dom.data(), sizeof(int) * h->blk_dom.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && h->d_ntiles)
        e = cudaMemcpy(h->d_ntiles, ntl.data(), sizeof(int4) * ntl.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_slot_dom, h->slot_dom.data(), sizeof(int) * NS, cudaMemcpyHostToDevice);
    // padding and not-yet-initialised cells are obstacles
    if (e == cudaSuccess) e = cudaMemset(h->flag, OBS, N);
    if (e == cudaSuccess) e = cudaMemset(h->mark, 0, N);
    if (e == cudaSuccess) e = cudaMemset(h->id, 0xff, 4 * N);
    if (e == cudaSuccess) e = cudaMemset(h->m, 0, 8 * N);
    if (e == cudaSuccess) e = cudaMemset(h->phi, 0, 8 * N);
    if (e == cudaSuccess) e = cudaMemset(h->phit, 0, 8 * N);
    if (e == cudaSuccess && h->phif) e = cudaMemset(h->phif, 0, 4 * N);
    if (e == cudaSuccess && h->phitf) e = cudaMemset(h->phitf, 0, 4 * N);
    if (e == cudaSuccess) e = cudaMemset(h->nrm, 0, 3 * N * (precision == FSL_P_FP64 ? 8 : 4));
    if (e == cudaSuccess) e = cudaMemset(h->nmask, 0, 4 * N);
    if (e == cudaSuccess) e = cudaMemset(h->pvc, 0, N * (precision == FSL_P_FP64 ? 8 : 4));
    if (e == cudaSuccess) e = cudaMemset(h->bbox, 0, 6 * 4 * NS);
    if (e == cudaSuccess) e = cudaMemset(h->rhoi, 0, 8 * N);
    if (e == cudaSuccess) e = cudaMemset(h->exs, 0, 8 * N);
    if (e == cudaSuccess) e = cudaMemset(h->f[0], 0, 19 * N * h->fbytes);
    if (e == cudaSuccess) e = cudaMemset(h->f[1], 0, 19 * N * h->fbytes);
    if (e == cudaSuccess) e = cudaMemset(h->pool, 0, 8 * n_domains);
    if (e == cudaSuccess) e = cudaMemset(h->nif, 0, 8 * n_domains);
    if (e == cudaSuccess) e = cudaMemset(h->trig, 0, sizeof(int) * (n_domains + 1));
    if (e == cudaSuccess) e = cudaMemset(h->status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->bar, 0, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(h->icount[0], 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->icount[1], 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->mcount, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->gcount, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->lcount, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->stepno, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->cstep, 0xff, 4 * N);
    if (e == cudaSuccess) e = cudaMemset(h->recv, 0xff, 4 * N);
    if (e == cudaSuccess) e = cudaMemset(h->icnt, 0, 8 * n_domains);
    if (e == cudaSuccess) e = cudaMemset(h->runs, 0, 16);
    if (e == cudaSuccess) e = cudaMemset(h->vfx, 0, 8 * NS);
    if (e == cudaSuccess) e = cudaMemset(h->vxfx, 0, 8 * NS);
    if (e == cudaSuccess) e = cudaMemset(h->vsfx, 0, 8 * NS);
    if (e == cudaSuccess) e = cudaMemset(h->ncells, 0, 8 * NS);
    if (e == cudaSuccess) e = cudaMemset(h->constp, 0, 4 * NS);
    // labelling: empty overlap hash, no marked bubble, no slot handed out
    if (e == cudaSuccess) e = cudaMemset(h->hkeys, 0xff, 8 * (size_t)hc);
    if (e == cudaSuccess) e = cudaMemset(h->hvals, 0, 8 * (size_t)hc);
    if (e == cudaSuccess) e = cudaMemset(h->aff, 0, 4 * NS);
    if (e == cudaSuccess) e = cudaMemset(h->naff, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->np, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->nnew, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->nhused, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->nused, 0, 4 * n_domains);
    if (e == cudaSuccess) e = cudaMemset(h->nfree, 0, 4 * n_domains);
    if (e != cudaSuccess) {
        fsl_destroy(h);
        return FSL_ERR_CUDA;
    }
    *out = h;
    return FSL_OK;
}

// Device address of page-locked host memory (which the GPU reads in place
// over the host link), or null for pageable memory.
static const void* mapped_host(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

fsl_status fsl_init_geometry(fsl_domain* h, int32_t d, const uint8_t* flags, const double* fill, const double* rho,
                             const double* u, int32_t on_device) {
    if (!h || d < 0 || d >= h->ndom || !flags || !fill || !rho || !u) return fail(h, FSL_ERR_ARG, "bad argument");
    if (h->stepped) return fail(h, FSL_ERR_ARG, "initialise every domain before the first step");
    const Dom& D = h->hdoms[d];
    const size_t n = (size_t)D.n;
    uint8_t* dfl = nullptr;
    double *dfi = nullptr, *drh = nullptr, *du = nullptr;
    if (!on_device) {
        CK(h, cudaStreamSynchronize(h->ls));   // queued work may still read the staging buffer
        const size_t bytes[4] = {n, 8 * n, 8 * n, 24 * n};
        void* parts[4];
        CK(h, staging(h, bytes, 4, parts));
        dfl = (uint8_t*)parts[0]; dfi = (double*)parts[1]; drh = (double*)parts[2]; du = (double*)parts[3];
        // on the library stream, so that the initialisation kernel below is
        // ordered after the copies (the stream is synchronised before return,
        // which also covers the caller's host buffers).  The cell types are
        // always staged (the kernel reads each cell's neighbours); fill level,
        // density and velocity in page-locked memory are read by the kernel
        // in place, once each, instead of being copied first.
        CK(h, cudaMemcpyAsync(dfl, flags, n, cudaMemcpyHostToDevice, h->ls));
        const void *mfi = mapped_host(fill), *mrh = mapped_host(rho), *mu = mapped_host(u);
        if (mfi && mrh && mu) {
            dfi = (double*)mfi; drh = (double*)mrh; du = (double*)mu;
        } else {
            CK(h, cudaMemcpyAsync(dfi, fill, 8 * n, cudaMemcpyHostToDevice, h->ls));
            CK(h, cudaMemcpyAsync(drh, rho, 8 * n, cudaMemcpyHostToDevice, h->ls));
            CK(h, cudaMemcpyAsync(du, u, 24 * n, cudaMemcpyHostToDevice, h->ls));
        }
    } else {
        dfl = (uint8_t*)flags; dfi = (double*)fill; drh = (double*)rho; du = (double*)u;
    }
    join_in(h);
    StepArgs A = step_args(h, 1 - h->cur);   // writes into f[cur]
    switch (h->precision) {
    case FSL_P_FP64: launch_init_state<double>(A, d, D.n, dfl, dfi, drh, du, h->ls); break;
    case FSL_P_FP32: launch_init_state<float>(A, d, D.n, dfl, dfi, drh, du, h->ls); break;
    case FSL_P_F16S: launch_init_state<__half>(A, d, D.n, dfl, dfi, drh, du, h->ls); break;
    default: launch_init_state<__nv_bfloat16>(A, d, D.n, dfl, dfi, drh, du, h->ls); break;
    }
    h->launches += 1;
    CK(h, cudaGetLastError());
    CK(h, cudaStreamSynchronize(h->ls));
    fsl_status st = latch(h);
    if (st != FSL_OK) return st;
    h->inited[d] = true;
    h->need_initial_ccl = true;
    join_out(h);
    return FSL_OK;
}

fsl_status fsl_set_bubble_source(fsl_domain* h, int32_t d, int64_t seed_cell, double extra0, double rate,
                                 int32_t const_pressure) {
    if (!h || d < 0 || d >= h->ndom) return fail(h, FSL_ERR_ARG, "bad domain");
    Dom& D = h->hdoms[d];
    if (seed_cell < 0 || seed_cell >= D.n) return fail(h, FSL_ERR_ARG, "seed cell outside the domain");
    if (h->stepped) return fail(h, FSL_ERR_ARG, "sources are attached before the first step");
    fsl_status st = ensure_initial(h);
    if (st != FSL_OK) return st;
    CK(h, cudaStreamSynchronize(h->ls));
    int slot = -1;
    CK(h, cudaMemcpy(&slot, h->id + D.off + seed_cell, sizeof(int), cudaMemcpyDeviceToHost));
    if (slot < 0) return fail(h, FSL_ERR_ARG, "seed cell is not a gas or interface cell");
    if (const_pressure) {
        int one = 1;
        CK(h, cudaMemcpy(h->constp + slot, &one, sizeof(int), cudaMemcpyHostToDevice));
        return FSL_OK;
    }
    if (D.seed >= 0) return fail(h, FSL_ERR_ARG, "one reservoir per domain");
    long long x0 = llrint(extra0 * 4294967296.0);
    long long vs = 0;
    CK(h, cudaMemcpy(&vs, h->vsfx + slot, sizeof(long long), cudaMemcpyDeviceToHost));
    vs += x0;
    CK(h, cudaMemcpy(h->vsfx + slot, &vs, sizeof(long long), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->vxfx + slot, &x0, sizeof(long long), cudaMemcpyHostToDevice));
    D.seed = (int)seed_cell;
    D.rate_fx = llrint(rate * 4294967296.0);
    CK(h, cudaMemcpy(h->d_doms + d, &D, sizeof(Dom), cudaMemcpyHostToDevice));
    return FSL_OK;
}

static void drop_graphs(fsl_domain* h);

namespace {

// The slab form needs the interface list in cell order; the tile-fused forms
// exist for the FP32-collide storage forms only (the FP64 cell needs more
// registers than two blocks per SM leave it).
bool form_usable(const fsl_domain* h, int f) {
    if (f == SC_SLAB) return order_effective(h) != 0;
    if (f == SC_TILE2 || f == SC_TILE4) return h->precision != FSL_P_FP64;
    return f >= 0 && f < SC_FORMS;
}

TuneKey tune_key(fsl_domain* h, int icount) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int lsize = 0;
    while ((1LL << (lsize + 1)) <= h->stride) ++lsize;
    return TuneKey{h->precision, h->ndom > 1 ? 1 : 0, sms, lsize, (int)(64LL * icount / std::max(1LL, h->stride))};
}

// One autotuning step: the next candidate form, its stream-collide kernel
// bracketed by events and timed (the call waits for it).  After the last
// candidate the fastest form is kept and recorded in the process cache.
fsl_status tune_step(fsl_domain* h) {
    if (h->tune_next == 0) {
        int ic = 0;
        CK(h, cudaMemcpyAsync(&ic, h->icount[h->cur], sizeof(int), cudaMemcpyDeviceToHost, h->ls));
        CK(h, cudaStreamSynchronize(h->ls));
        const TuneKey key = tune_key(h, ic);
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            h->form = it->second;
            h->tuning = false;
            h->tune_source = 2;
            return FSL_OK;   // no step taken: the caller runs it with the cached form
        }
    }
    while (h->tune_next < kTuneSteps && !form_usable(h, kTuneSeq[h->tune_next])) ++h->tune_next;
    const int f = kTuneSeq[h->tune_next];
    if (!h->tev[0]) {
        CK(h, cudaEventCreate(&h->tev[0]));
        CK(h, cudaEventCreate(&h->tev[1]));
    }
    StepArgs A = step_args(h, h->cur);
    CK(h, cudaEventRecord(h->tev[0], h->ls));
    launch_k1(h, A, h->ls, nullptr, nullptr, f);
    CK(h, cudaEventRecord(h->tev[1], h->ls));
    CK(h, launch_conv(h, A, h->ls, f));
    h->launches += kernels_per_step(f);
    h->cur = 1 - h->cur;
    CK(h, cudaEventSynchronize(h->tev[1]));
    float ms = 0.f;
    CK(h, cudaEventElapsedTime(&ms, h->tev[0], h->tev[1]));
    if (h->tune_ms[f] == 0.0 || ms < h->tune_ms[f]) h->tune_ms[f] = ms;
    ++h->tune_next;
    while (h->tune_next < kTuneSteps && !form_usable(h, kTuneSeq[h->tune_next])) ++h->tune_next;
    if (h->tune_next == kTuneSteps) {
        int best = SC_SPLIT;
        for (int g = 0; g < SC_FORMS; ++g)
            if (h->tune_ms[g] > 0.0 && h->tune_ms[g] < h->tune_ms[best]) best = g;
        h->form = best;
        h->tuning = false;
        h->tune_source = 1;
        int ic = 0;
        CK(h, cudaMemcpyAsync(&ic, h->icount[h->cur], sizeof(int), cudaMemcpyDeviceToHost, h->ls));
        CK(h, cudaStreamSynchronize(h->ls));
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[tune_key(h, ic)] = best;
        drop_graphs(h);
    }
    return FSL_OK;
}

}  // namespace

fsl_status fsl_step(fsl_domain* h, int64_t nsteps) {
    if (!h || nsteps < 0) return fail(h, FSL_ERR_ARG, "bad argument");
    fsl_status st = ensure_initial(h);
    if (st != FSL_OK) return st;
    h->stepped = true;
    join_in(h);
    int64_t k = 0;
    // autotuning steps first (each a real step of the simulation)
    while (h->tuning && k < nsteps) {
        const int before = h->cur;
        st = tune_step(h);
        if (st != FSL_OK) return st;
        if (h->cur != before) ++k;   // a cache hit decides without a step
    }
    if (k == nsteps) {
        CK(h, cudaGetLastError());
        join_out(h);
        return FSL_OK;
    }
    nsteps -= k;
    k = 0;
    if (!h->graphs) {
        // direct launches
        for (; k < nsteps; ++k) {
            StepArgs A = step_args(h, h->cur);
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (h->timing) {
                auto ev = next_events(h);
                e0 = ev.first;
                e1 = ev.second;
            }
            h->launches += enqueue_main(h, A, e0, e1, nullptr, h->timing);
            h->cur = 1 - h->cur;
        }
    } else if (h->timing) {
        for (; k < nsteps; ++k) {
            st = launch_graph(h, 2);
            if (st != FSL_OK) return st;
            h->cur = 1 - h->cur;
        }
    } else {
        for (; k + 2 <= nsteps; k += 2) {
            st = launch_graph(h, 0);
            if (st != FSL_OK) return st;
        }
        if (k < nsteps) {
            st = launch_graph(h, 1);
            if (st != FSL_OK) return st;
            h->cur = 1 - h->cur;
        }
    }
    CK(h, cudaGetLastError());
    join_out(h);
    return FSL_OK;
}

fsl_status fsl_sync(fsl_domain* h) {
    if (!h) return FSL_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->ls));
    if (h->timing && h->evused > 0) {
        double tot = 0.0;
        for (size_t k = 0; k + 1 < h->evused; k += 2) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, h->evpool[k], h->evpool[k + 1]);
            tot += ms;
        }
        h->k1_ms = tot;
        // direct mode, three phase events per step: two at the end of the
        // stream-collide kernel (timed from its start), then the end of the
        // conversion kernel (timed from the end of the stream-collide kernel)
        if (h->phused >= 3 && h->phused == 3 * (h->evused / 2)) {
            for (int k = 0; k < 4; ++k) h->phase_ms[k] = 0.0;
            for (size_t n = 0; n < h->evused / 2; ++n) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, h->evpool[2 * n], h->evpool[2 * n + 1]);
                h->phase_ms[0] += ms;
                for (int k = 0; k < 2; ++k) {
                    cudaEventElapsedTime(&ms, h->evpool[2 * n], h->phpool[3 * n + k]);
                    h->phase_ms[1 + k] += ms;
                }
                cudaEventElapsedTime(&ms, h->evpool[2 * n + 1], h->phpool[3 * n + 2]);
                h->phase_ms[3] += ms;
            }
        }
        h->evused = 0;
        h->phused = 0;
    }
    return latch(h);
}

fsl_status fsl_set_timing(fsl_domain* h, int32_t on) {
    if (!h) return FSL_ERR_ARG;
    h->timing = on != 0;
    h->k1_ms = 0.0;
    h->evused = 0;
    h->phused = 0;
    return FSL_OK;
}

double fsl_stream_collide_ms(const fsl_domain* h) { return h ? h->k1_ms : 0.0; }

fsl_status fsl_phase_ms(const fsl_domain* h, double* out) {
    if (!h || !out) return FSL_ERR_ARG;
    for (int k = 0; k < 4; ++k) out[k] = h->phase_ms[k];
    return FSL_OK;
}

static void drop_graphs(fsl_domain* h);

fsl_status fsl_set_limits(fsl_domain* h, int64_t ccl_max_iter, int64_t barrier_polls, int32_t barrier_absent) {
    if (!h) return FSL_ERR_ARG;
    if (ccl_max_iter < 0 || ccl_max_iter > INT_MAX || barrier_polls < 0 || barrier_polls > INT_MAX ||
        (barrier_absent != 0 && barrier_absent != 1))
        return fail(h, FSL_ERR_ARG, "bad limit");
    CK(h, cudaStreamSynchronize(h->ls));
    h->ccl_cap = ccl_max_iter > 0 ? (int)ccl_max_iter : (1 << 24);
    h->spins = barrier_polls > 0 ? (int)barrier_polls : (1 << 22);
    h->bar_extra = barrier_absent;
    drop_graphs(h);   // the step graphs hold the old values in their kernel parameters
    return FSL_OK;
}

static void drop_graphs(fsl_domain* h) {
    for (int k = 0; k < 2; ++k)
        for (int j = 0; j < 3; ++j)
            if (h->graph[k][j]) { cudaGraphExecDestroy(h->graph[k][j]); h->graph[k][j] = nullptr; }
    for (int k = 0; k < 2; ++k)
        if (h->timed_src[k]) { cudaGraphDestroy(h->timed_src[k]); h->timed_src[k] = nullptr; }
}

fsl_status fsl_set_stream_form(fsl_domain* h, int32_t form) {
    if (!h || form < -1 || form >= SC_FORMS) return fail(h, FSL_ERR_ARG, "bad stream-collide form");
    if (form >= 0 && !form_usable(h, form))
        return fail(h, FSL_ERR_ARG, form == SC_SLAB ? "the slab form needs the interface list in cell order"
                                                    : "the tile-fused forms need FP32 or 16-bit storage");
    CK(h, cudaStreamSynchronize(h->ls));
    if (form < 0) {
        // autotune again from the next step on (the process cache is consulted first)
        h->tuning = true;
        h->tune_next = 0;
        for (int f = 0; f < SC_FORMS; ++f) h->tune_ms[f] = 0.0;
        h->tune_source = 0;
    } else {
        h->form = form;
        h->tuning = false;
        h->tune_source = 3;
    }
    drop_graphs(h);   // the step graphs hold the previous kernel
    return FSL_OK;
}

fsl_status fsl_tuning(const fsl_domain* h, double* ms_per_form, int32_t* form, int32_t* source) {
    if (!h) return FSL_ERR_ARG;
    if (ms_per_form)
        for (int f = 0; f < SC_FORMS; ++f) ms_per_form[f] = h->tune_ms[f];
    if (form) *form = h->tuning ? -1 : h->form;
    if (source) *source = h->tune_source;
    return FSL_OK;
}

fsl_status fsl_forget_tuning(void) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache.clear();
    return FSL_OK;
}

int32_t fsl_stream_form(const fsl_domain* h) { return h ? h->form : -1; }

fsl_status fsl_set_interface_order(fsl_domain* h, int32_t mode) {
    if (!h || mode < -1 || mode > 1) return fail(h, FSL_ERR_ARG, "bad interface-order mode");
    CK(h, cudaStreamSynchronize(h->ls));
    h->order_mode = mode;
    if (h->form == SC_SLAB && !order_effective(h)) h->form = SC_SPLIT;   // the slab form needs the order
    drop_graphs(h);
    return FSL_OK;
}

int32_t fsl_interface_order(const fsl_domain* h) { return h ? order_effective(h) : -1; }

fsl_status fsl_set_graphs(fsl_domain* h, int32_t on) {
    if (!h) return FSL_ERR_ARG;
    h->graphs = on != 0;
    return FSL_OK;
}

int64_t fsl_kernel_launches(const fsl_domain* h) { return h ? h->launches : 0; }

int64_t fsl_labelling_runs(fsl_domain* h) {
    if (!h) return -1;
    long long r = 0;
    if (cudaStreamSynchronize(h->ls) != cudaSuccess) return -1;
    if (cudaMemcpy(&r, h->runs, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    return r;
}

int64_t fsl_relabelled_bubbles(fsl_domain* h) {
    if (!h) return -1;
    long long r = 0;
    if (cudaStreamSynchronize(h->ls) != cudaSuccess) return -1;
    if (cudaMemcpy(&r, h->runs + 1, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    return r;
}

const char* fsl_last_error(const fsl_domain* h) { return h ? h->err.c_str() : "null handle"; }

static fsl_status compute_minidx(fsl_domain* h, int d) {
    const Dom& D = h->hdoms[d];
    CK(h, cudaMemsetAsync(h->minidx + D.slot_off, 0x7f, 4 * (size_t)D.slot_cap, h->ls));
    launch_export_minid(h->id, D.off, D.n, h->minidx, h->ls);
    h->launches += 1;
    return FSL_OK;
}

fsl_status fsl_bubbles(fsl_domain* h, int32_t d, fsl_bubble* out, int64_t cap, int64_t* count) {
    if (!h || d < 0 || d >= h->ndom || !count) return fail(h, FSL_ERR_ARG, "bad argument");
    fsl_status st = ensure_initial(h);
    if (st != FSL_OK) return st;
    join_in(h);
    st = compute_minidx(h, d);
    if (st != FSL_OK) return st;
    const Dom& D = h->hdoms[d];
    // only the slots handed out so far (the domain's high-water mark) hold bubbles
    int used = 0;
    CK(h, cudaMemcpyAsync(&used, h->nused + d, sizeof(int), cudaMemcpyDeviceToHost, h->ls));
    CK(h, cudaStreamSynchronize(h->ls));
    const size_t C = (size_t)std::max(0, std::min(used, D.slot_cap));
    std::vector<long long> vfx(C), vxfx(C), vsfx(C), nc(C);
    std::vector<int> cp(C), mi(C);
    CK(h, cudaMemcpyAsync(vfx.data(), h->vfx + D.slot_off, 8 * C, cudaMemcpyDeviceToHost, h->ls));
    CK(h, cudaMemcpyAsync(vxfx.data(), h->vxfx + D.slot_off, 8 * C, cudaMemcpyDeviceToHost, h->ls));
    CK(h, cudaMemcpyAsync(vsfx.data(), h->vsfx + D.slot_off, 8 * C, cudaMemcpyDeviceToHost, h->ls));
    CK(h, cudaMemcpyAsync(nc.data(), h->ncells + D.slot_off, 8 * C, cudaMemcpyDeviceToHost, h->ls));
    CK(h, cudaMemcpyAsync(cp.data(), h->constp + D.slot_off, 4 * C, cudaMemcpyDeviceToHost, h->ls));
    CK(h, cudaMemcpyAsync(mi.data(), h->minidx + D.slot_off, 4 * C, cudaMemcpyDeviceToHost, h->ls));
    CK(h, cudaStreamSynchronize(h->ls));
    std::vector<fsl_bubble> rec;
    const double unit = 2.3283064365386962890625e-10;
    const double p0 = 1.0 / 3.0;
    for (size_t s = 0; s < C; ++s) {
        if (nc[s] <= 0) continue;
        fsl_bubble b;
        memset(&b, 0, sizeof(b));
        b.id = mi[s];
        double V = (double)(vfx[s] + vxfx[s]) * unit;
        double Vs = (double)vsfx[s] * unit;
        b.volume = V;
        b.init_volume = Vs;
        b.n_cells = nc[s];
        b.const_pressure = cp[s];
        b.extra_volume = (double)vxfx[s] * unit;
        if (cp[s]) b.pressure = p0;
        else if (V <= 1e-3) b.pressure = p0;
        else b.pressure = (Vs / V) * p0;
        rec.push_back(b);
    }
    std::sort(rec.begin(), rec.end(), [](const fsl_bubble& a, const fsl_bubble& b) { return a.id < b.id; });
    *count = (int64_t)rec.size();
    if (out) {
        for (int64_t k = 0; k < cap && k < (int64_t)rec.size(); ++k) out[k] = rec[(size_t)k];
    }
    join_out(h);
    return latch(h);
}

fsl_status fsl_fields(fsl_domain* h, int32_t d, uint32_t mask, void* const* dst, int32_t on_device) {
    if (!h || d < 0 || d >= h->ndom || (mask & ~127u) || (mask && !dst)) return fail(h, FSL_ERR_ARG, "bad argument");
    fsl_status st = ensure_initial(h);
    if (st != FSL_OK) return st;
    join_in(h);
    const Dom& D = h->hdoms[d];
    const size_t n = (size_t)D.n;
    if (mask & FSL_F_ID) {
        st = compute_minidx(h, d);
        if (st != FSL_OK) return st;
    }
    // device targets: the caller's buffers, or slices of the staging buffer
    // copied out after (the previous calls on the handle's stream, which may
    // read the staging buffer, are done: every call ends synchronised)
    size_t sizes[7] = {n, 8 * n, 8 * n, 8 * n, 8 * n, 24 * n, 152 * n};
    void* dev[7] = {nullptr};
    if (on_device) {
        int k = 0;
        for (int bit = 0; bit < 7; ++bit)
            if (mask & (1u << bit)) dev[bit] = dst[k++];
    } else {
        size_t want[7];
        void* parts[7];
        int m = 0;
        for (int bit = 0; bit < 7; ++bit)
            if (mask & (1u << bit)) want[m++] = sizes[bit];
        CK(h, staging(h, want, m, parts));
        m = 0;
        for (int bit = 0; bit < 7; ++bit)
            if (mask & (1u << bit)) dev[bit] = parts[m++];
    }
    if (mask & (FSL_F_FLAGS | FSL_F_FILL | FSL_F_MASS | FSL_F_ID)) {
        launch_export_cells(h->flag, h->phi, h->phif, h->m, h->id, h->minidx, D.off, D.n, (uint8_t*)dev[0], (double*)dev[1],
                            (double*)dev[2], (long long*)dev[3], nullptr, h->ls);
        h->launches += 1;
    }
    if (mask & (FSL_F_RHO | FSL_F_U | FSL_F_PDF)) {
        switch (h->precision) {
        case FSL_P_FP64: launch_export_pdf<double>(h->f[h->cur], h->stride, D.off, D.n, (double*)dev[6], (double*)dev[4], (double*)dev[5], h->ls); break;
        case FSL_P_FP32: launch_export_pdf<float>(h->f[h->cur], h->stride, D.off, D.n, (double*)dev[6], (double*)dev[4], (double*)dev[5], h->ls); break;
        case FSL_P_F16S: launch_export_pdf<__half>(h->f[h->cur], h->stride, D.off, D.n, (double*)dev[6], (double*)dev[4], (double*)dev[5], h->ls); break;
        default: launch_export_pdf<__nv_bfloat16>(h->f[h->cur], h->stride, D.off, D.n, (double*)dev[6], (double*)dev[4], (double*)dev[5], h->ls); break;
        }
        h->launches += 1;
    }
    CK(h, cudaGetLastError());
    if (!on_device) {
        int k = 0;
        for (int bit = 0; bit < 7; ++bit) {
            if (!(mask & (1u << bit))) continue;
            CK(h, cudaMemcpyAsync(dst[k], dev[bit], sizes[bit], cudaMemcpyDeviceToHost, h->ls));
            ++k;
        }
    }
    CK(h, cudaStreamSynchronize(h->ls));
    join_out(h);
    return latch(h);
}

fsl_status fsl_cell_counts(fsl_domain* h, int32_t d, int64_t* counts) {
    if (!h || d < 0 || d >= h->ndom || !counts) return fail(h, FSL_ERR_ARG, "bad argument");
    join_in(h);
    const Dom& D = h->hdoms[d];
    CK(h, cudaMemsetAsync(h->counts, 0, 64, h->ls));
    launch_export_cells(h->flag, h->phi, h->phif, h->m, h->id, h->minidx, D.off, D.n, nullptr, nullptr, nullptr, nullptr,
                        h->counts, h->ls);
    h->launches += 1;
    long long c[8];
    CK(h, cudaMemcpyAsync(c, h->counts, 64, cudaMemcpyDeviceToHost, h->ls));
    CK(h, cudaStreamSynchronize(h->ls));
    for (int k = 0; k < 5; ++k) counts[k] = c[k];
    join_out(h);
    return latch(h);
}

fsl_status fsl_total_mass(fsl_domain* h, int32_t d, double* mass) {
    if (!h || d < 0 || d >= h->ndom || !mass) return fail(h, FSL_ERR_ARG, "bad argument");
    fsl_status st = ensure_initial(h);
    if (st != FSL_OK) return st;
    join_in(h);
    const Dom& D = h->hdoms[d];
    const long long nb = ((long long)D.n + FSL_BLOCK - 1) / FSL_BLOCK;
    switch (h->precision) {
    case FSL_P_FP64: launch_mass_partials<double>(h->f[h->cur], h->flag, h->m, h->stride, D.off, D.n, h->mass_part, h->ls); break;
    case FSL_P_FP32: launch_mass_partials<float>(h->f[h->cur], h->flag, h->m, h->stride, D.off, D.n, h->mass_part, h->ls); break;
    case FSL_P_F16S: launch_mass_partials<__half>(h->f[h->cur], h->flag, h->m, h->stride, D.off, D.n, h->mass_part, h->ls); break;
    default: launch_mass_partials<__nv_bfloat16>(h->f[h->cur], h->flag, h->m, h->stride, D.off, D.n, h->mass_part, h->ls); break;
    }
    h->launches += 1;
    CK(h, cudaGetLastError());
    std::vector<double> part((size_t)nb);
    long long pool = 0;
    CK(h, cudaMemcpyAsync(part.data(), h->mass_part, 8 * (size_t)nb, cudaMemcpyDeviceToHost, h->ls));
    CK(h, cudaMemcpyAsync(&pool, h->pool + d, 8, cudaMemcpyDeviceToHost, h->ls));
    CK(h, cudaStreamSynchronize(h->ls));
    double t = 0.0;
    for (double v : part) t += v;
    // excess mass pooled and not yet shared out (fixed point 2^-40)
    *mass = t + (double)pool * 9.094947017729282379150390625e-13;
    join_out(h);
    return latch(h);
}

fsl_status fsl_destroy(fsl_domain* h) {
    if (!h) return FSL_ERR_ARG;
    if (h->ls) cudaStreamSynchronize(h->ls);
    for (int k = 0; k < 2; ++k)
        for (int j = 0; j < 3; ++j)
            if (h->graph[k][j]) cudaGraphExecDestroy(h->graph[k][j]);
    for (int k = 0; k < 2; ++k)
        if (h->timed_src[k]) cudaGraphDestroy(h->timed_src[k]);
    for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
    for (cudaEvent_t e : h->tev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : h->phpool) cudaEventDestroy(e);
    for (void* p : h->allocs) cudaFree(p);
    if (h->stage) cudaFree(h->stage);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->ls) cudaStreamDestroy(h->ls);
    if (h->ls2) cudaStreamDestroy(h->ls2);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    delete h;
    return FSL_OK;
}

}  // extern "C"
