// pic_api.cu -- host implementation of the libpic C ABI (include/pic.h).
//
// Owns the context: device buffers (through the caller's allocator callback
// or cudaMalloc), the box and species tables, the frame pool of the mixed
// form, the per-step CUDA graphs, stage timing, and the device status word.
// Every entry point returns a pic_status; no exception crosses the ABI.
#include "pic.h"
#include "pic_internal.cuh"
#include "plain.cuh"

#include <cuda.h>  // pointer-attribute types only; the driver call goes through cudaGetDriverEntryPointByVersion

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include <mutex>
#include <map>

using namespace pic;

namespace {

struct PlainSpecies {
    double *x = nullptr, *y = nullptr, *z = nullptr, *ux = nullptr, *uy = nullptr, *uz = nullptr,
           *w = nullptr;
    int* pid = nullptr;
    int64_t n = 0, cap = 0;
};

struct PlainBox {
    double *E = nullptr, *B = nullptr, *J = nullptr;
    std::vector<PlainSpecies> sp;
};

constexpr int kStageTimers = 4;  // push, frames, yee, whole step

}  // namespace

struct pic_ctx {
    // configuration
    int precision = PIC_PRECISION_MIXED;
    std::vector<pic_grid> grids;
    int nboxes = 0;
    double h[3] = {1, 1, 1};
    double dt = 0;
    std::vector<pic_species> sp;
    pic_options opt{};
    std::vector<double> rho_bg;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int nsm = 0;
    size_t smem_optin = 0;
    // errors
    std::string err;
    pic_status poisoned = PIC_OK;
    // allocations
    std::vector<void*> allocs;
    unsigned* status_d = nullptr;
    double* diag_d = nullptr;
    double* rho_d = nullptr;
    int* ioff_d = nullptr;  // scratch ints for read-back offsets
    int64_t ioff_cap = 0;
    void* stage_d = nullptr;
    size_t stage_bytes = 0;
    // mixed form
    int LX = 4, LY = 4, LZ = 4, S = 64, log2S = 6, threads = 64;
    int guard = 1;  // field guard cells below the interior: 2 when a species has the PCS shape
    int push_grid = 0;
    std::vector<BoxDev> boxes_h;
    BoxDev* boxes_d = nullptr;
    CUtensorMap* tmaps_d = nullptr;  // [nboxes][2] E, B tile maps of the push
    int* sc_box_d = nullptr;
    int* items_d = nullptr;
    int* yee_off_d = nullptr;
    int yee_nblocks = 0;
    float *E_all = nullptr, *B_all = nullptr, *J_all = nullptr;
    int64_t field_floats = 0;  // per field, all boxes (3 components each)
    int nsc = 0, nlists = 0;
    int *count = nullptr, *nframes = nullptr, *narrive = nullptr, *abase = nullptr;
    int* foff[2] = {nullptr, nullptr};
    int* ftab[2] = {nullptr, nullptr};
    int *cell = nullptr, *pid = nullptr;
    float *ox = nullptr, *oy = nullptr, *oz = nullptr, *ux = nullptr, *uy = nullptr, *uz = nullptr,
          *w = nullptr;
    int *free_stack = nullptr, *free_top = nullptr, *released = nullptr;
    int64_t pool_cap = 0;  // frames
    int64_t frames_used = 0;
    int mv_cap = 0;
    int *mv_count = nullptr, *mv_dest = nullptr, *mv_rank = nullptr, *mv_cell = nullptr,
        *mv_pid = nullptr;
    float *mv_ox = nullptr, *mv_oy = nullptr, *mv_oz = nullptr, *mv_ux = nullptr, *mv_uy = nullptr,
          *mv_uz = nullptr, *mv_w = nullptr;
    int4 *blk_sums = nullptr, *blk_offs = nullptr, *totals = nullptr;
    int* work_counter = nullptr;
    int* step_ctr = nullptr;           // device step count, read by the push for its sort passes
    long long* step_no = nullptr;      // device: steps taken since creation (antenna time)
    int64_t steps_done = 0;            // host: steps enqueued since creation
    int64_t host_direct = 0;           // load / read calls that converted page-locked host arrays in place
    int* abs_off_d = nullptr;          // [nboxes + 1] block offsets of the y absorber
    int abs_nblocks = 0;
    bool any_antenna = false;
    float* shift_scratch = nullptr;    // moving window: copy of one box's field
    int64_t shift_scratch_floats = 0;
    int* rot_scratch = nullptr;        // moving window: copies of count, nframes, foff
    int sort_every = kDefaultSortEvery;
    unsigned* wmax_bits = nullptr;     // [kMaxSpecies] device
    float wmax[kMaxSpecies] = {};      // host copy: largest |weight| per species
    int parity = 0;
    bool prepared = false;
    // subdomain slab (pic_set_subdomain): the two face messages of migrants
    bool sub_z = false;
    char* mig = nullptr;
    int64_t mig_bytes = 0;
    int mig_cap = 0;
    int next_stage = 0;  // pic_step_stage: the stage expected next (0 = a step starts)
    // in-library autotuning (pic_options sc = 0,0,0 and/or threads_per_sc = 0)
    bool tune_sc = false, tune_threads = false, tune_pending = false;
    int tune_trials = 0;  // configurations timed by the last tuning (0: given or cached)
    std::vector<int64_t> id_next;  // per (box, species)
    int64_t total_particles = 0;
    // graphs (one per frame-table parity); each holds four event-record
    // nodes at the stage boundaries, re-pointed at fresh events per replay
    // when stage timing is on
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaGraphNode_t evnode[2][4] = {};
    cudaEvent_t placeholder[8] = {};
    bool graph_failed = false;
    // fused field update (pic_options.field_update 0): a second field buffer
    // pair; a pair of steps goes first -> second -> first.  The tables, push
    // maps and Yee maps of the second pair mirror those of the first.
    bool fused_ready = false;   // pairs of steps take the fused update
    bool field_chosen = false;  // the field update was chosen (at the first step)
    float *E_alt = nullptr, *B_alt = nullptr;
    BoxDev* boxes_alt_d = nullptr;
    CUtensorMap* tmaps_alt_d = nullptr;  // [nboxes][2] push tile maps over E_alt, B_alt
    CUtensorMap* ymaps_d = nullptr;      // [2][nboxes][3] plane maps of k_yee_fused: E, B, J of either pair
    int* fused_off_d = nullptr;
    int fused_nblocks = 0;
    int64_t fused_steps = 0;
    // graphs of a pair of steps, one per frame-table parity of its first step
    cudaGraph_t pgraph[2] = {nullptr, nullptr};
    cudaGraphExec_t pgexec[2] = {nullptr, nullptr};
    cudaGraphNode_t pevnode[2][8] = {};
    // plain form
    std::vector<PlainBox> pboxes;
    // stage timing
    bool timing = false;
    std::vector<cudaEvent_t> events;  // kStageTimers+? per recorded step: 4 boundaries
    int64_t ev_steps = 0;             // steps with events pending
    double acc_ms[kStageTimers] = {0, 0, 0, 0};
    int64_t timed_steps = 0;
};

namespace {

pic_status fail(pic_ctx* c, pic_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) {
        c->err = buf;
        if (st != PIC_ERR_ARG && c->poisoned == PIC_OK)
            c->poisoned = st;
    }
    return st;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e__ = (call);                                                         \
        if (e__ != cudaSuccess)                                                           \
            return fail(c, PIC_ERR_CUDA, "%s failed: %s (%s:%d)", #call,                 \
                        cudaGetErrorString(e__), __FILE__, __LINE__);                     \
    } while (0)

#define CKS(expr)                     \
    do {                              \
        pic_status s__ = (expr);      \
        if (s__ != PIC_OK)            \
            return s__;               \
    } while (0)

void* raw_alloc(pic_ctx* c, size_t bytes)
{
    if (bytes == 0)
        bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (c->opt.dev_alloc) {
        p = c->opt.dev_alloc(bytes, c->opt.alloc_ud);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p)
        c->allocs.push_back(p);
    return p;
}

void raw_free(pic_ctx* c, void* p)
{
    if (!p)
        return;
    auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
    if (it != c->allocs.end())
        c->allocs.erase(it);
    if (c->opt.dev_free)
        c->opt.dev_free(p, c->opt.alloc_ud);
    else if (!c->opt.dev_alloc)
        cudaFree(p);
}

template <class T>
pic_status dalloc(pic_ctx* c, T** out, int64_t count, bool zero = true)
{
    void* p = raw_alloc(c, sizeof(T) * (size_t)std::max<int64_t>(count, 1));
    if (!p)
        return fail(c, PIC_ERR_OOM, "device allocation of %lld bytes failed",
                    (long long)(sizeof(T) * count));
    if (zero) {
        cudaError_t e = cudaMemsetAsync(p, 0, sizeof(T) * (size_t)std::max<int64_t>(count, 1),
                                        c->stream);
        if (e != cudaSuccess)
            return fail(c, PIC_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
    *out = static_cast<T*>(p);
    return PIC_OK;
}

pic_status check_ctx(pic_ctx* c)
{
    if (!c)
        return PIC_ERR_ARG;
    if (c->poisoned != PIC_OK)
        return PIC_ERR_STATE;
    return PIC_OK;
}

void destroy_graphs(pic_ctx* c)
{
    for (int p = 0; p < 2; ++p) {
        if (c->gexec[p])
            cudaGraphExecDestroy(c->gexec[p]);
        if (c->graph[p])
            cudaGraphDestroy(c->graph[p]);
        c->gexec[p] = nullptr;
        c->graph[p] = nullptr;
        if (c->pgexec[p])
            cudaGraphExecDestroy(c->pgexec[p]);
        if (c->pgraph[p])
            cudaGraphDestroy(c->pgraph[p]);
        c->pgexec[p] = nullptr;
        c->pgraph[p] = nullptr;
    }
}

pic_status ensure_stage(pic_ctx* c, size_t bytes)
{
    if (bytes <= c->stage_bytes)
        return PIC_OK;
    CK(cudaStreamSynchronize(c->stream));
    raw_free(c, c->stage_d);
    c->stage_d = nullptr;
    c->stage_bytes = 0;
    void* p = raw_alloc(c, bytes);
    if (!p)
        return fail(c, PIC_ERR_OOM, "staging allocation of %zu bytes failed", bytes);
    c->stage_d = p;
    c->stage_bytes = bytes;
    return PIC_OK;
}

// Device address of the host range [p, p + bytes) when all of it lies in one
// page-locked host allocation mapped into this device's address space
// (cudaHostAlloc / cudaHostRegister, e.g. torch pin_memory); nullptr
// otherwise, and then the caller stages through device memory.  The particle
// conversion kernels read and write such buffers directly over the host
// link, which saves the staging buffer and a copy.  The allocation's extent
// comes from the driver (cuPointerGetAttribute, reached through the runtime's
// entry-point query, so libpic needs no link to the driver library); when
// that query is unavailable the range is not used directly.
const void* host_range_on_device(const void* p, size_t bytes)
{
    if (!p || bytes == 0)
        return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer)
        return nullptr;
    using GetAttr = CUresult (*)(void*, CUpointer_attribute, CUdeviceptr);
    static GetAttr get_attr = [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            fn = nullptr;
        }
        return reinterpret_cast<GetAttr>(fn);
    }();
    if (!get_attr)
        return nullptr;
    const CUdeviceptr dp = reinterpret_cast<CUdeviceptr>(a.devicePointer);
    CUdeviceptr start = 0;
    size_t size = 0;
    if (get_attr(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, dp) != CUDA_SUCCESS ||
        get_attr(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, dp) != CUDA_SUCCESS)
        return nullptr;
    if (dp < start || dp - start > size || bytes > size - (dp - start))
        return nullptr;
    return a.devicePointer;
}

pic_status ensure_ioff(pic_ctx* c, int64_t n)
{
    if (n <= c->ioff_cap)
        return PIC_OK;
    CK(cudaStreamSynchronize(c->stream));
    raw_free(c, c->ioff_d);
    c->ioff_d = nullptr;
    CKS(dalloc(c, &c->ioff_d, n, false));
    c->ioff_cap = n;
    return PIC_OK;
}

pic_status status_check(pic_ctx* c)
{
    CK(cudaStreamSynchronize(c->stream));
    unsigned st = 0;
    CK(cudaMemcpy(&st, c->status_d, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (st == 0)
        return PIC_OK;
    if (st & ST_FRAME_POOL)
        return fail(c, PIC_ERR_FRAME_POOL,
                    "frame pool exhausted (%lld frames); create the context with a larger "
                    "pool_frames",
                    (long long)c->pool_cap);
    if (st & ST_CAPACITY)
        return fail(c, PIC_ERR_CAPACITY,
                    "more than %d particles changed supercell in one step; raise move_capacity",
                    c->mv_cap);
    if (st & ST_TIMEOUT)
        return fail(c, PIC_ERR_TIMEOUT, "a device-side wait timed out");
    return fail(c, PIC_ERR_PARTICLE, "a particle got a non-finite or superluminal momentum");
}

// ------------------------------------------------------------ mixed form

pic_status insert_mixed(pic_ctx* c, int box, int species, int64_t m, const double* sx, const double* su,
                        const double* sw, int id_base, const int64_t* ids);
pic_status autotune(pic_ctx* c);
pic_status prepare_fused(pic_ctx* c);
pic_status choose_field_update(pic_ctx* c);
pic_status status_check(pic_ctx* c);

// alt: the step reads its fields from the second buffer pair (the second
// step of a fused pair)
StepDev make_step(const pic_ctx* c, int parity, bool alt = false)
{
    StepDev d{};
    d.LX = c->LX;
    d.LY = c->LY;
    d.LZ = c->LZ;
    d.S = c->S;
    d.log2S = c->log2S;
    d.guard = c->guard;
    d.nboxes = c->nboxes;
    d.nsc = c->nsc;
    d.nspecies = (int)c->sp.size();
    d.nlists = c->nlists;
    d.dt = (float)c->dt;
    for (int a = 0; a < 3; ++a)
        d.move[a] = (float)(c->dt / c->h[a]);
    d.boxes = alt ? c->boxes_alt_d : c->boxes_d;
    d.tmaps = alt ? c->tmaps_alt_d : c->tmaps_d;
    d.sc_box = c->sc_box_d;
    d.items = c->items_d;
    const double V = c->h[0] * c->h[1] * c->h[2];
    for (size_t s = 0; s < c->sp.size(); ++s) {
        const pic_species& p = c->sp[s];
        SpeciesDev& q = d.sp[s];
        q.eps = (float)(p.charge * c->dt / (2.0 * p.mass));
        for (int a = 0; a < 3; ++a)
            q.jcoef[a] = (float)(-p.charge * c->h[a] / (V * c->dt));
        q.q = (float)p.charge;
        q.m = (float)p.mass;
        q.shape = p.shape;
        q.mobile = p.mobile;
        q.ec = p.gather == PIC_GATHER_ENERGY;
        float jmax = std::max({std::fabs(q.jcoef[0]), std::fabs(q.jcoef[1]), std::fabs(q.jcoef[2])});
        q.cbound = jmax * c->wmax[s] * 1.0001f;  // headroom for FP32 rounding
    }
    d.cell = c->cell;
    d.ox = c->ox;
    d.oy = c->oy;
    d.oz = c->oz;
    d.ux = c->ux;
    d.uy = c->uy;
    d.uz = c->uz;
    d.w = c->w;
    d.pid = c->pid;
    d.count = c->count;
    d.nframes = c->nframes;
    d.foff = c->foff[parity];
    d.ftab = c->ftab[parity];
    d.foff_next = c->foff[parity ^ 1];
    d.ftab_next = c->ftab[parity ^ 1];
    d.narrive = c->narrive;
    d.abase = c->abase;
    d.free_stack = c->free_stack;
    d.free_top = c->free_top;
    d.released = c->released;
    d.pool_frames = (int)c->pool_cap;
    d.mv_cap = c->mv_cap;
    d.mv_count = c->mv_count;
    d.mv_dest = c->mv_dest;
    d.mv_rank = c->mv_rank;
    d.mv_cell = c->mv_cell;
    d.mv_ox = c->mv_ox;
    d.mv_oy = c->mv_oy;
    d.mv_oz = c->mv_oz;
    d.mv_ux = c->mv_ux;
    d.mv_uy = c->mv_uy;
    d.mv_uz = c->mv_uz;
    d.mv_w = c->mv_w;
    d.mv_pid = c->mv_pid;
    d.mig = c->mig;
    d.mig_bytes = c->mig_bytes;
    d.mig_cap = c->mig_cap;
    d.blk_sums = c->blk_sums;
    d.blk_offs = c->blk_offs;
    d.totals = c->totals;
    d.work_counter = c->work_counter;
    d.step_ctr = c->step_ctr;
    d.step_no = c->step_no;
    d.sort_every = c->sort_every;
    d.status = c->status_d;
    d.wmax_bits = c->wmax_bits;
    return d;
}

template <class T>
pic_status grow_copy(pic_ctx* c, T** arr, int64_t old_n, int64_t new_n)
{
    T* p = nullptr;
    CKS(dalloc(c, &p, new_n, false));
    if (*arr && old_n > 0)
        CK(cudaMemcpyAsync(p, *arr, sizeof(T) * old_n, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    raw_free(c, *arr);
    *arr = p;
    return PIC_OK;
}

pic_status read_free_top(pic_ctx* c, int* top)
{
    CK(cudaMemcpyAsync(top, c->free_top, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

// Grow the frame pool to at least `frames` frames, keeping every frame's
// contents and the free stack.
pic_status ensure_pool(pic_ctx* c, int64_t frames)
{
    if (frames <= c->pool_cap)
        return PIC_OK;
    int64_t new_cap = std::max<int64_t>(frames, c->pool_cap + c->pool_cap / 2);
    if (new_cap * (int64_t)c->S >= (int64_t)1 << 40 || new_cap >= ((int64_t)1 << 31) - 1)
        return fail(c, PIC_ERR_OOM, "frame pool of %lld frames is too large", (long long)new_cap);
    destroy_graphs(c);
    int top = 0;
    if (c->pool_cap > 0)
        CKS(read_free_top(c, &top));
    const int64_t oldS = c->pool_cap * c->S, newS = new_cap * c->S;
    CKS(grow_copy(c, &c->cell, oldS, newS));
    CKS(grow_copy(c, &c->ox, oldS, newS));
    CKS(grow_copy(c, &c->oy, oldS, newS));
    CKS(grow_copy(c, &c->oz, oldS, newS));
    CKS(grow_copy(c, &c->ux, oldS, newS));
    CKS(grow_copy(c, &c->uy, oldS, newS));
    CKS(grow_copy(c, &c->uz, oldS, newS));
    CKS(grow_copy(c, &c->w, oldS, newS));
    if (c->opt.track_ids)
        CKS(grow_copy(c, &c->pid, oldS, newS));
    // frame tables: both parities hold at most every frame of the pool
    CKS(grow_copy(c, &c->ftab[0], c->pool_cap, new_cap));
    CKS(grow_copy(c, &c->ftab[1], c->pool_cap, new_cap));
    CKS(grow_copy(c, &c->released, 0, new_cap));
    // free stack: keep [0, top), push the new frames
    CKS(grow_copy(c, &c->free_stack, top, new_cap));
    std::vector<int> fresh((size_t)(new_cap - c->pool_cap));
    for (size_t i = 0; i < fresh.size(); ++i)
        fresh[i] = (int)(new_cap - 1 - (int64_t)i);
    CK(cudaMemcpyAsync(c->free_stack + top, fresh.data(), sizeof(int) * fresh.size(),
                       cudaMemcpyHostToDevice, c->stream));
    int new_top = top + (int)fresh.size();
    CK(cudaMemcpyAsync(c->free_top, &new_top, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->pool_cap = new_cap;
    return PIC_OK;
}

// Capacity of the buffer of particles that change supercell (also the load
// staging of converted particles).  Its contents never outlive a step.
pic_status ensure_mv(pic_ctx* c, int64_t cap)
{
    if (cap <= c->mv_cap)
        return PIC_OK;
    if (cap > INT32_MAX / 2)
        cap = INT32_MAX / 2;
    destroy_graphs(c);
    CK(cudaStreamSynchronize(c->stream));
    int** ints[] = {&c->mv_dest, &c->mv_rank, &c->mv_cell};
    float** floats[] = {&c->mv_ox, &c->mv_oy, &c->mv_oz, &c->mv_ux, &c->mv_uy, &c->mv_uz, &c->mv_w};
    for (auto p : ints) {
        raw_free(c, *p);
        *p = nullptr;
        CKS(dalloc(c, p, cap, false));
    }
    for (auto p : floats) {
        raw_free(c, *p);
        *p = nullptr;
        CKS(dalloc(c, p, cap, false));
    }
    if (c->opt.track_ids) {
        raw_free(c, c->mv_pid);
        c->mv_pid = nullptr;
        CKS(dalloc(c, &c->mv_pid, cap, false));
    }
    c->mv_cap = (int)cap;
    return PIC_OK;
}

cudaError_t record(cudaEvent_t e, cudaStream_t s, bool external)
{
    return external ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

YeePlan yee_plan(const pic_ctx* c)
{
    return YeePlan{c->boxes_d, c->yee_off_d, c->nboxes, c->yee_nblocks, (float)c->dt,
                   {(float)(1.0 / c->h[0]), (float)(1.0 / c->h[1]), (float)(1.0 / c->h[2])},
                   c->step_no, c->dt, {c->h[0], c->h[1], c->h[2]}, c->abs_off_d, c->abs_nblocks,
                   c->any_antenna ? 1 : 0, c->guard, c->sub_z ? 1 : 0};
}

// The fused field update of one step: from the first buffer pair into the
// second (src 0) or back (src 1).
FusedPlan fused_plan(const pic_ctx* c, int src)
{
    return FusedPlan{src ? c->boxes_alt_d : c->boxes_d, src ? c->boxes_d : c->boxes_alt_d,
                     c->ymaps_d + (size_t)src * 3 * c->nboxes, c->fused_off_d, c->fused_nblocks, c->status_d};
}

// One stage of the mixed-form step (PIC_STAGE_*) on frame-table parity
// `parity`; the Yee stages run one part of the field update each.  fsrc 0 /
// 1: a step of a fused pair, whose fields are read from the first / second
// buffer pair (the push and frames stages only; its field update is
// launch_yee_fused).
pic_status enqueue_stage(pic_ctx* c, int stage, int parity, int fsrc = -1)
{
    const StepDev d = make_step(c, parity, fsrc == 1);
    switch (stage) {
    case PIC_STAGE_PUSH:
        CK(cudaMemsetAsync(c->work_counter, 0, sizeof(int), c->stream));
        CK(cudaMemsetAsync(c->J_all, 0, sizeof(float) * c->field_floats, c->stream));
        if (c->mig) {  // the face messages start empty (their capacity word stays)
            CK(cudaMemsetAsync(c->mig, 0, sizeof(int), c->stream));
            CK(cudaMemsetAsync(c->mig + c->mig_bytes, 0, sizeof(int), c->stream));
        }
        CK(launch_push_deposit(d, c->threads, c->push_grid, c->stream));
        return PIC_OK;
    case PIC_STAGE_FRAMES:
        CK(launch_frame_plan(d, c->stream));
        CK(launch_frame_apply(d, 4 * c->nsm, c->stream));
        return PIC_OK;
    default:
        CK(launch_yee_mixed_part(yee_plan(c), stage - PIC_STAGE_B_FIRST, c->stream));
        return PIC_OK;
    }
}

// One step; fsrc -1: in place, 0 / 1: the first / second step of a fused
// pair (fields read from the first / second buffer pair, written to the
// other).
pic_status enqueue_step_mixed(pic_ctx* c, int parity, cudaEvent_t* ev, bool external = false, int fsrc = -1)
{
    if (ev)
        CK(record(ev[0], c->stream, external));
    CKS(enqueue_stage(c, PIC_STAGE_PUSH, parity, fsrc));
    if (ev)
        CK(record(ev[1], c->stream, external));
    CKS(enqueue_stage(c, PIC_STAGE_FRAMES, parity, fsrc));
    if (ev)
        CK(record(ev[2], c->stream, external));
    if (fsrc >= 0) {
        CK(launch_yee_fused(yee_plan(c), fused_plan(c, fsrc), c->stream));
    } else {
        for (int st = PIC_STAGE_B_FIRST; st <= PIC_STAGE_B_SECOND; ++st)
            CKS(enqueue_stage(c, st, parity));
    }
    if (ev)
        CK(record(ev[3], c->stream, external));
    return PIC_OK;
}

// Two steps with the fused field update: first pair -> second -> first, so
// that the state is back in the first buffer pair; ev: 8 events (or null).
pic_status enqueue_pair_mixed(pic_ctx* c, int parity, cudaEvent_t* ev, bool external = false)
{
    CKS(enqueue_step_mixed(c, parity, ev, external, 0));
    return enqueue_step_mixed(c, parity ^ 1, ev ? ev + 4 : nullptr, external, 1);
}

// Before the first step: room in the frame pool for one step of growth,
// a move buffer sized for the particle count.
pic_status prepare_mixed(pic_ctx* c)
{
    if (c->prepared)
        return PIC_OK;
    int top = 0;
    CKS(read_free_top(c, &top));
    c->frames_used = c->pool_cap - top;
    int64_t want = c->opt.pool_frames > 0
                       ? c->opt.pool_frames
                       : c->frames_used + c->frames_used / 4 + c->nlists / 4 + 1024;
    CKS(ensure_pool(c, want));
    int64_t mv = c->opt.move_capacity > 0 ? c->opt.move_capacity
                                          : std::max<int64_t>(1 << 20, c->total_particles / 6);
    CKS(ensure_mv(c, mv));
    int per_sm = 0;
    CK(configure_push(c->LX, c->LY, c->LZ, c->threads, c->guard, &per_sm));
    c->push_grid = std::max(1, per_sm) * c->nsm;
    CKS(prepare_fused(c));
    c->prepared = true;
    return PIC_OK;
}

// Capture one step per frame-table parity.  Any failure leaves the context
// on eager launches (same kernels, same order).
pic_status capture_graphs(pic_ctx* c)
{
    if (c->gexec[0] || c->graph_failed)
        return PIC_OK;
    for (cudaEvent_t& e : c->placeholder)
        if (!e)
            CK(cudaEventCreate(&e));
    for (int p = 0; p < 2; ++p) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            c->graph_failed = true;
            return PIC_OK;
        }
        pic_status st = enqueue_step_mixed(c, p, c->placeholder, true);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (st != PIC_OK) {
            if (g)
                cudaGraphDestroy(g);
            return st;
        }
        bool ok = e == cudaSuccess && g;
        if (ok) {
            size_t n = 0;
            ok = cudaGraphGetNodes(g, nullptr, &n) == cudaSuccess;
            std::vector<cudaGraphNode_t> nodes(n);
            ok = ok && cudaGraphGetNodes(g, nodes.data(), &n) == cudaSuccess;
            int found = 0;
            for (size_t i = 0; ok && i < n; ++i) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess || t != cudaGraphNodeTypeEventRecord)
                    continue;
                cudaEvent_t ev = nullptr;
                if (cudaGraphEventRecordNodeGetEvent(nodes[i], &ev) != cudaSuccess)
                    continue;
                for (int k = 0; k < 4; ++k)
                    if (ev == c->placeholder[k]) {
                        c->evnode[p][k] = nodes[i];
                        ++found;
                    }
            }
            ok = ok && found == 4 && cudaGraphInstantiate(&c->gexec[p], g, 0) == cudaSuccess;
        }
        if (!ok) {
            cudaGetLastError();
            if (g)
                cudaGraphDestroy(g);
            destroy_graphs(c);
            c->graph_failed = true;
            return PIC_OK;
        }
        c->graph[p] = g;
    }
    return PIC_OK;
}

// Capture a pair of steps with the fused field update per frame-table
// parity of its first step (after capture_graphs succeeded).  A failure
// leaves pairs on eager launches.
pic_status capture_pair_graphs(pic_ctx* c)
{
    if (!c->fused_ready || c->pgexec[0] || c->graph_failed || !c->gexec[0])
        return PIC_OK;
    for (int p = 0; p < 2; ++p) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            c->graph_failed = true;
            return PIC_OK;
        }
        pic_status st = enqueue_pair_mixed(c, p, c->placeholder, true);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (st != PIC_OK) {
            if (g)
                cudaGraphDestroy(g);
            return st;
        }
        bool ok = e == cudaSuccess && g;
        int found = 0;
        if (ok) {
            size_t n = 0;
            ok = cudaGraphGetNodes(g, nullptr, &n) == cudaSuccess;
            std::vector<cudaGraphNode_t> nodes(n);
            ok = ok && cudaGraphGetNodes(g, nodes.data(), &n) == cudaSuccess;
            for (size_t i = 0; ok && i < n; ++i) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess || t != cudaGraphNodeTypeEventRecord)
                    continue;
                cudaEvent_t ev = nullptr;
                if (cudaGraphEventRecordNodeGetEvent(nodes[i], &ev) != cudaSuccess)
                    continue;
                for (int k = 0; k < 8; ++k)
                    if (ev == c->placeholder[k]) {
                        c->pevnode[p][k] = nodes[i];
                        ++found;
                    }
            }
        }
        ok = ok && found == 8 && cudaGraphInstantiate(&c->pgexec[p], g, 0) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            if (g)
                cudaGraphDestroy(g);
            destroy_graphs(c);
            c->graph_failed = true;
            return PIC_OK;
        }
        c->pgraph[p] = g;
    }
    return PIC_OK;
}

pic_status launch_pair_graph(pic_ctx* c, int p, cudaEvent_t* ev)
{
    for (int k = 0; k < 8; ++k)
        CK(cudaGraphExecEventRecordNodeSetEvent(c->pgexec[p], c->pevnode[p][k], ev ? ev[k] : c->placeholder[k]));
    CK(cudaGraphLaunch(c->pgexec[p], c->stream));
    return PIC_OK;
}

pic_status launch_graph(pic_ctx* c, int p, cudaEvent_t* ev)
{
    for (int k = 0; k < 4; ++k)
        CK(cudaGraphExecEventRecordNodeSetEvent(c->gexec[p], c->evnode[p][k], ev ? ev[k] : c->placeholder[k]));
    CK(cudaGraphLaunch(c->gexec[p], c->stream));
    return PIC_OK;
}

// ------------------------------------------------------------ stage timing

pic_status harvest_events(pic_ctx* c)
{
    if (c->ev_steps == 0)
        return PIC_OK;
    CK(cudaStreamSynchronize(c->stream));
    for (int64_t s = 0; s < c->ev_steps; ++s) {
        cudaEvent_t* e = &c->events[(size_t)s * 4];
        float a = 0, b = 0, d = 0, t = 0;
        CK(cudaEventElapsedTime(&a, e[0], e[1]));
        CK(cudaEventElapsedTime(&b, e[1], e[2]));
        CK(cudaEventElapsedTime(&d, e[2], e[3]));
        CK(cudaEventElapsedTime(&t, e[0], e[3]));
        c->acc_ms[0] += a;
        c->acc_ms[1] += b;
        c->acc_ms[2] += d;
        c->acc_ms[3] += t;
        c->timed_steps += 1;
    }
    c->ev_steps = 0;
    return PIC_OK;
}

// Events for the next `steps` steps (4 each, contiguous).
pic_status step_events(pic_ctx* c, cudaEvent_t** out, int steps = 1)
{
    const int64_t kMaxPending = 512;
    if (c->ev_steps + steps > kMaxPending)
        CKS(harvest_events(c));
    size_t need = (size_t)(c->ev_steps + steps) * 4;
    while (c->events.size() < need) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        c->events.push_back(e);
    }
    *out = &c->events[(size_t)c->ev_steps * 4];
    c->ev_steps += steps;
    return PIC_OK;
}

// ------------------------------------------------------------ plain form

pic_status plain_grow(pic_ctx* c, PlainSpecies& s, int64_t need)
{
    if (need <= s.cap)
        return PIC_OK;
    int64_t cap = std::max<int64_t>(need, s.cap + s.cap / 2);
    double** arrs[] = {&s.x, &s.y, &s.z, &s.ux, &s.uy, &s.uz, &s.w};
    for (auto a : arrs)
        CKS(grow_copy(c, a, s.n, cap));
    if (c->opt.track_ids)
        CKS(grow_copy(c, &s.pid, s.n, cap));
    s.cap = cap;
    return PIC_OK;
}

PlainPushArgs plain_args(const pic_ctx* c, int box, int species)
{
    const pic_grid& g = c->grids[box];
    const PlainBox& b = c->pboxes[box];
    const PlainSpecies& s = b.sp[species];
    const pic_species& p = c->sp[species];
    PlainPushArgs a{};
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.n = s.n;
    a.E = b.E;
    a.B = b.B;
    a.J = b.J;
    a.x = s.x;
    a.y = s.y;
    a.z = s.z;
    a.ux = s.ux;
    a.uy = s.uy;
    a.uz = s.uz;
    a.w = s.w;
    const double V = c->h[0] * c->h[1] * c->h[2];
    a.eps = p.charge * c->dt / (2.0 * p.mass);
    a.ec = p.gather == PIC_GATHER_ENERGY;
    for (int d = 0; d < 3; ++d) {
        a.jcoef[d] = -p.charge * c->h[d] / (V * c->dt);
        a.move[d] = c->dt / c->h[d];
    }
    a.status = c->status_d;
    return a;
}

PlainYeeArgs plain_yee_args(const pic_ctx* c, int box)
{
    const pic_grid& g = c->grids[box];
    const PlainBox& b = c->pboxes[box];
    PlainYeeArgs a{};
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.E = b.E;
    a.B = b.B;
    a.J = b.J;
    for (int d = 0; d < 3; ++d)
        a.ih[d] = 1.0 / c->h[d];
    return a;
}

pic_status enqueue_step_plain(pic_ctx* c, cudaEvent_t* ev)
{
    if (ev)
        CK(cudaEventRecord(ev[0], c->stream));
    for (int b = 0; b < c->nboxes; ++b) {
        const pic_grid& g = c->grids[b];
        int64_t nc = (int64_t)g.nx * g.ny * g.nz;
        CK(cudaMemsetAsync(c->pboxes[b].J, 0, sizeof(double) * 3 * nc, c->stream));
        for (size_t s = 0; s < c->sp.size(); ++s)
            if (c->sp[s].mobile)
                CK(launch_plain_push(plain_args(c, b, (int)s), c->sp[s].shape, c->stream));
    }
    if (ev) {
        CK(cudaEventRecord(ev[1], c->stream));
        CK(cudaEventRecord(ev[2], c->stream));
    }
    for (int b = 0; b < c->nboxes; ++b)
        CK(launch_plain_yee(plain_yee_args(c, b), c->dt, c->stream));
    if (ev)
        CK(cudaEventRecord(ev[3], c->stream));
    return PIC_OK;
}

bool valid_box(const pic_ctx* c, int box) { return box >= 0 && box < c->nboxes; }

int ilog2(int v)
{
    int r = 0;
    while ((1 << r) < v)
        ++r;
    return r;
}

}  // namespace

// ============================================================ C ABI

namespace {

using TensorEncode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

TensorEncode tensor_encoder()
{
    static TensorEncode encode = [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            fn = nullptr;
        }
        return reinterpret_cast<TensorEncode>(fn);
    }();
    return encode;
}

// One box's padded field array F (three components) as a 4D tensor (x, y,
// z, component) with the given box extents.  Reads past the array come back
// as zeros.
pic_status encode_field_map(pic_ctx* c, CUtensorMap* map, const BoxDev& bd, float* F, int bx, int by, int bz,
                            int box)
{
    TensorEncode encode = tensor_encoder();
    if (!encode)
        return fail(c, PIC_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[4] = {(cuuint64_t)bd.px, (cuuint64_t)bd.py, (cuuint64_t)bd.pz, 3};
    const cuuint64_t strides[3] = {(cuuint64_t)bd.px * 4, (cuuint64_t)bd.px * bd.py * 4,
                                   (cuuint64_t)padded_cells(bd) * 4};
    const cuuint32_t ext[4] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 3};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, F, dims, strides, ext, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(c, PIC_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for box %d", (int)r, box);
    return PIC_OK;
}

// TMA descriptors of the push's E/B tile loads, one per box and field, over
// the fields of the box table `boxes`: box = the tile (row pitch px, ty
// rows, tz planes, 3 components), so that one load brings a supercell's
// three components into shared memory.
pic_status encode_tile_maps(pic_ctx* c, const std::vector<BoxDev>& boxes, CUtensorMap** out)
{
    int bpx = 0, bty = 0, btz = 0;
    push_tile_box(c->LX, c->LY, c->LZ, c->guard, &bpx, &bty, &btz);
    std::vector<CUtensorMap> maps((size_t)2 * c->nboxes);
    for (int b = 0; b < c->nboxes; ++b)
        for (int f = 0; f < 2; ++f)
            CKS(encode_field_map(c, &maps[2 * b + f], boxes[b], f == 0 ? boxes[b].E : boxes[b].B, bpx, bty,
                                 btz, b));
    CKS(dalloc(c, out, 2 * c->nboxes, false));
    CK(cudaMemcpyAsync(*out, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

pic_status encode_tile_maps(pic_ctx* c) { return encode_tile_maps(c, c->boxes_h, &c->tmaps_d); }

// The host box table with the fields of the second buffer pair.
std::vector<BoxDev> alt_boxes(const pic_ctx* c)
{
    std::vector<BoxDev> alt = c->boxes_h;
    for (BoxDev& b : alt) {
        b.E = c->E_alt + (b.E - c->E_all);
        b.B = c->B_alt + (b.B - c->B_all);
    }
    return alt;
}

// The second field buffer pair of the fused field update, its box table,
// its push tile maps and the E plane maps of k_yee_fused over both pairs
// (pic_options.field_update 0; not for subdomain slabs, which step by
// stages).
pic_status prepare_fused(pic_ctx* c)
{
    if (c->fused_ready || c->field_chosen || c->opt.field_update == PIC_FIELD_UPDATE_IN_PLACE || c->sub_z ||
        c->precision != PIC_PRECISION_MIXED)
        return PIC_OK;
    CKS(dalloc(c, &c->E_alt, c->field_floats));
    CKS(dalloc(c, &c->B_alt, c->field_floats));
    const std::vector<BoxDev> alt = alt_boxes(c);
    CKS(dalloc(c, &c->boxes_alt_d, c->nboxes, false));
    CK(cudaMemcpyAsync(c->boxes_alt_d, alt.data(), sizeof(BoxDev) * c->nboxes, cudaMemcpyHostToDevice,
                       c->stream));
    CKS(encode_tile_maps(c, alt, &c->tmaps_alt_d));
    std::vector<CUtensorMap> ymaps((size_t)6 * c->nboxes);
    std::vector<int> off(c->nboxes + 1, 0);
    for (int b = 0; b < c->nboxes; ++b) {
        for (int src = 0; src < 2; ++src) {
            const BoxDev& bd = src ? alt[b] : c->boxes_h[b];
            float* F[3] = {bd.E, bd.B, bd.J};
            for (int f = 0; f < 3; ++f)
                CKS(encode_field_map(c, &ymaps[((size_t)src * c->nboxes + b) * 3 + f], bd, F[f], kFusedEX,
                                     kFusedTY + 3, 1, b));
        }
        off[b + 1] = off[b] + fused_blocks(c->boxes_h[b].nx, c->boxes_h[b].ny, c->boxes_h[b].nz);
    }
    CK(configure_yee_fused());
    CKS(dalloc(c, &c->ymaps_d, 6 * c->nboxes, false));
    CKS(dalloc(c, &c->fused_off_d, c->nboxes + 1, false));
    CK(cudaMemcpyAsync(c->ymaps_d, ymaps.data(), sizeof(CUtensorMap) * ymaps.size(), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(c->fused_off_d, off.data(), sizeof(int) * (c->nboxes + 1), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->fused_nblocks = off[c->nboxes];
    c->fused_ready = true;
    c->field_chosen = true;
    if (c->opt.field_update == PIC_FIELD_UPDATE_AUTO)
        CKS(choose_field_update(c));
    return PIC_OK;
}

// PIC_FIELD_UPDATE_AUTO: one fused update (first pair -> second, which
// leaves the state alone) against the in-place kernels run on a copy of the
// fields in the second pair, three times each after a first run of each; the
// faster by its best time stays.  Only J is written besides the second pair
// (an antenna adds into it), and the next push zeroes J first.
pic_status choose_field_update(pic_ctx* c)
{
    YeePlan onto_alt = yee_plan(c);
    onto_alt.boxes = c->boxes_alt_d;
    const FusedPlan f = fused_plan(c, 0);
    cudaEvent_t ev[4];
    for (cudaEvent_t& e : ev)
        CK(cudaEventCreate(&e));
    float best_fused = 1e30f, best_in_place = 1e30f;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
        const size_t bytes = sizeof(float) * c->field_floats;
        if ((err = cudaEventRecord(ev[0], c->stream)) != cudaSuccess ||
            (err = launch_yee_fused(yee_plan(c), f, c->stream)) != cudaSuccess ||
            (err = cudaEventRecord(ev[1], c->stream)) != cudaSuccess ||
            (err = cudaMemcpyAsync(c->E_alt, c->E_all, bytes, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess ||
            (err = cudaMemcpyAsync(c->B_alt, c->B_all, bytes, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess ||
            (err = cudaEventRecord(ev[2], c->stream)) != cudaSuccess ||
            (err = launch_yee_mixed_plan(onto_alt, c->stream)) != cudaSuccess ||
            (err = cudaEventRecord(ev[3], c->stream)) != cudaSuccess ||
            (err = cudaStreamSynchronize(c->stream)) != cudaSuccess)
            break;
        float tf = 0, ti = 0;
        if ((err = cudaEventElapsedTime(&tf, ev[0], ev[1])) != cudaSuccess ||
            (err = cudaEventElapsedTime(&ti, ev[2], ev[3])) != cudaSuccess)
            break;
        if (rep > 0) {
            best_fused = std::min(best_fused, tf);
            best_in_place = std::min(best_in_place, ti);
        }
    }
    for (cudaEvent_t e : ev)
        cudaEventDestroy(e);
    CK(err);
    CKS(status_check(c));
    if (best_fused < best_in_place)
        return PIC_OK;
    // the in-place kernels: drop the second pair
    c->fused_ready = false;
    raw_free(c, c->E_alt);
    raw_free(c, c->B_alt);
    c->E_alt = c->B_alt = nullptr;
    return PIC_OK;
}

// Copy the host box table (open-y options included) to the device and
// rebuild the absorber's block table; a change of the absorber's launch
// shape drops the captured graphs.
pic_status upload_boxes(pic_ctx* c)
{
    std::vector<int> off(c->nboxes + 1, 0);
    for (int b = 0; b < c->nboxes; ++b)
        off[b + 1] = off[b] + absorber_blocks(c->boxes_h[b]);
    bool ant = false;
    for (int b = 0; b < c->nboxes; ++b)
        ant = ant || c->boxes_h[b].oy.ant_j >= 0;
    if (off[c->nboxes] != c->abs_nblocks || ant != c->any_antenna)
        destroy_graphs(c);
    c->abs_nblocks = off[c->nboxes];
    c->any_antenna = ant;
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpyAsync(c->boxes_d, c->boxes_h.data(), sizeof(BoxDev) * c->nboxes,
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->abs_off_d, off.data(), sizeof(int) * (c->nboxes + 1),
                       cudaMemcpyHostToDevice, c->stream));
    if (c->boxes_alt_d) {
        const std::vector<BoxDev> alt = alt_boxes(c);
        CK(cudaMemcpyAsync(c->boxes_alt_d, alt.data(), sizeof(BoxDev) * c->nboxes, cudaMemcpyHostToDevice,
                           c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

}  // namespace


extern "C" {

pic_status pic_create(const pic_grid* grids, int32_t nboxes, const double dx[3], double dt,
                      const pic_species* sp, int32_t nspecies, const pic_options* opt,
                      pic_ctx** out)
{
    if (!out)
        return PIC_ERR_ARG;
    *out = nullptr;
    if (!grids || nboxes < 1 || !dx || !sp || nspecies < 1 || nspecies > kMaxSpecies)
        return PIC_ERR_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt))
        return PIC_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(dx[a] > 0.0) || !std::isfinite(dx[a]))
            return PIC_ERR_ARG;
    for (int b = 0; b < nboxes; ++b)
        if (grids[b].nx < 4 || grids[b].ny < 4 || grids[b].nz < 4)
            return PIC_ERR_ARG;
    for (int s = 0; s < nspecies; ++s)
        if (!(sp[s].mass > 0.0) || !std::isfinite(sp[s].charge) || sp[s].shape < 1 || sp[s].shape > 3 ||
            (sp[s].gather != PIC_GATHER_MOMENTUM && sp[s].gather != PIC_GATHER_ENERGY))
            return PIC_ERR_ARG;
    // no particle may cross half a cell per step (|v| < c), and the Yee
    // scheme must be stable
    const double courant = 1.0 / std::sqrt(1.0 / (dx[0] * dx[0]) + 1.0 / (dx[1] * dx[1]) +
                                           1.0 / (dx[2] * dx[2]));
    if (!(dt < 0.5 * std::min({dx[0], dx[1], dx[2]})) || !(dt < courant))
        return PIC_ERR_CFL;

    pic_ctx* c = new (std::nothrow) pic_ctx();
    if (!c)
        return PIC_ERR_OOM;
    pic_options o{};
    if (opt)
        o = *opt;
    c->opt = o;
    c->precision = o.precision;
    c->grids.assign(grids, grids + nboxes);
    c->nboxes = nboxes;
    for (int a = 0; a < 3; ++a)
        c->h[a] = dx[a];
    c->dt = dt;
    c->sp.assign(sp, sp + nspecies);
    c->rho_bg.assign(nboxes, 0.0);
    c->id_next.assign((size_t)nboxes * nspecies, 0);
    if ((c->precision != PIC_PRECISION_FP64_PLAIN && c->precision != PIC_PRECISION_MIXED) ||
        o.sort_every < 0 || o.field_update < PIC_FIELD_UPDATE_AUTO || o.field_update > PIC_FIELD_UPDATE_FUSED) {
        delete c;
        return PIC_ERR_ARG;
    }

    auto bail = [&](pic_status st) {
        pic_destroy(c);
        return st;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        return bail(PIC_ERR_CUDA);
    }
    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    c->smem_optin = (size_t)optin;
    if (o.stream) {
        c->stream = static_cast<cudaStream_t>(o.stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return bail(PIC_ERR_CUDA);
        }
        c->own_stream = true;
    }
    if (dalloc(c, &c->status_d, 1) != PIC_OK || dalloc(c, &c->diag_d, 4) != PIC_OK)
        return bail(PIC_ERR_OOM);
    int64_t max_cells = 0;
    for (int b = 0; b < nboxes; ++b)
        max_cells = std::max<int64_t>(max_cells, (int64_t)grids[b].nx * grids[b].ny * grids[b].nz);
    if (dalloc(c, &c->rho_d, max_cells, false) != PIC_OK)
        return bail(PIC_ERR_OOM);

    if (c->precision == PIC_PRECISION_FP64_PLAIN) {
        for (int s = 0; s < nspecies; ++s)
            if (sp[s].shape == 3)
                return bail(PIC_ERR_ARG);  // the plain form has CIC and TSC only
        c->pboxes.resize(nboxes);
        for (int b = 0; b < nboxes; ++b) {
            int64_t nc = (int64_t)grids[b].nx * grids[b].ny * grids[b].nz;
            PlainBox& pb = c->pboxes[b];
            if (dalloc(c, &pb.E, 3 * nc) != PIC_OK || dalloc(c, &pb.B, 3 * nc) != PIC_OK ||
                dalloc(c, &pb.J, 3 * nc) != PIC_OK)
                return bail(PIC_ERR_OOM);
            pb.sp.resize(nspecies);
        }
    } else {
        int sc[3] = {o.sc[0], o.sc[1], o.sc[2]};
        // zeros: tuned by the library at the first step (tune_candidates);
        // until then the particles sit in 4 x 4 x 4 supercells / the
        // supercell's default thread count
        c->tune_sc = sc[0] == 0 && sc[1] == 0 && sc[2] == 0;
        c->tune_threads = o.threads_per_sc == 0;
        c->tune_pending = c->tune_sc || c->tune_threads;
        if (c->tune_sc)
            sc[0] = sc[1] = sc[2] = 4;
        c->LX = sc[0];
        c->LY = sc[1];
        c->LZ = sc[2];
        c->S = sc[0] * sc[1] * sc[2];
        c->log2S = ilog2(c->S);
        c->threads = o.threads_per_sc > 0 ? o.threads_per_sc : (c->S >= 256 ? 256 : 128);
        c->sort_every = o.sort_every > 0 ? o.sort_every : kDefaultSortEvery;
        for (int s = 0; s < nspecies; ++s)
            if (sp[s].shape == 3)
                c->guard = 2;
        if ((1 << c->log2S) != c->S || !push_supported(c->LX, c->LY, c->LZ, c->threads, c->guard))
            return bail(PIC_ERR_ARG);
        if (push_smem_bytes(c->LX, c->LY, c->LZ, c->threads, c->guard) > c->smem_optin)
            return bail(PIC_ERR_ARG);
        // boxes
        c->boxes_h.resize(nboxes);
        int64_t floats = 0;
        int nsc = 0;
        std::vector<int> yee_off(nboxes + 1, 0);
        for (int b = 0; b < nboxes; ++b) {
            const pic_grid& g = grids[b];
            if (g.nx % c->LX || g.ny % c->LY || g.nz % c->LZ)
                return bail(PIC_ERR_ARG);
            if (c->guard == 2 && (g.nx < 8 || g.ny < 8 || g.nz < 8))  // one periodic image per guard cell
                return bail(PIC_ERR_ARG);
            BoxDev& bd = c->boxes_h[b];
            bd.nx = g.nx;
            bd.ny = g.ny;
            bd.nz = g.nz;
            // guards: TSC/CIC tiles reach 1 cell below and 3 (x, 16-byte rows) /
            // 2 (y, z) above; PCS tiles 2 below and 6 (x) / 3 (y, z) above
            const int G = c->guard;
            bd.gx = bd.gy = bd.gz = G;
            bd.px = g.nx + (G == 1 ? 4 : 8);
            bd.py = g.ny + (G == 1 ? 3 : 5);
            bd.pz = g.nz + (G == 1 ? 3 : 5);
            bd.nscx = g.nx / c->LX;
            bd.nscy = g.ny / c->LY;
            bd.nscz = g.nz / c->LZ;
            bd.sc_base = nsc;
            bd.oy = OpenYDev{};
            bd.oy.ant_j = -1;
            nsc += bd.nscx * bd.nscy * bd.nscz;
            floats += 3 * padded_cells(bd);
            yee_off[b + 1] = yee_off[b] + ((g.nx + 31) / 32) * ((g.ny + 7) / 8) * (g.nz / kYeeCellsZ);
        }
        c->nsc = nsc;
        c->nlists = nsc * nspecies;
        c->field_floats = floats;
        c->yee_nblocks = yee_off[nboxes];
        if (dalloc(c, &c->E_all, floats) != PIC_OK || dalloc(c, &c->B_all, floats) != PIC_OK ||
            dalloc(c, &c->J_all, floats) != PIC_OK)
            return bail(PIC_ERR_OOM);
        int64_t off = 0;
        std::vector<int> sc_box(nsc);
        for (int b = 0; b < nboxes; ++b) {
            BoxDev& bd = c->boxes_h[b];
            bd.E = c->E_all + off;
            bd.B = c->B_all + off;
            bd.J = c->J_all + off;
            off += 3 * padded_cells(bd);
            for (int i = 0; i < bd.nscx * bd.nscy * bd.nscz; ++i)
                sc_box[bd.sc_base + i] = b;
        }
        std::vector<int> items(nsc);
        for (int i = 0; i < nsc; ++i)
            items[i] = i;
        const int nblk = (c->nlists + 4095) / 4096;
        if (dalloc(c, &c->boxes_d, nboxes, false) != PIC_OK || dalloc(c, &c->sc_box_d, nsc, false) != PIC_OK ||
            dalloc(c, &c->items_d, nsc, false) != PIC_OK || dalloc(c, &c->yee_off_d, nboxes + 1, false) != PIC_OK ||
            dalloc(c, &c->count, c->nlists) != PIC_OK || dalloc(c, &c->nframes, c->nlists) != PIC_OK ||
            dalloc(c, &c->narrive, c->nlists) != PIC_OK || dalloc(c, &c->abase, c->nlists) != PIC_OK ||
            dalloc(c, &c->foff[0], c->nlists) != PIC_OK || dalloc(c, &c->foff[1], c->nlists) != PIC_OK ||
            dalloc(c, &c->free_top, 1) != PIC_OK || dalloc(c, &c->mv_count, 1) != PIC_OK ||
            dalloc(c, &c->blk_sums, nblk) != PIC_OK || dalloc(c, &c->blk_offs, nblk) != PIC_OK ||
            dalloc(c, &c->totals, 1) != PIC_OK || dalloc(c, &c->work_counter, 1) != PIC_OK ||
            dalloc(c, &c->step_ctr, 1) != PIC_OK || dalloc(c, &c->step_no, 1) != PIC_OK ||
            dalloc(c, &c->abs_off_d, nboxes + 1) != PIC_OK || dalloc(c, &c->wmax_bits, kMaxSpecies) != PIC_OK)
            return bail(PIC_ERR_OOM);
        if (cudaMemcpyAsync(c->boxes_d, c->boxes_h.data(), sizeof(BoxDev) * nboxes,
                            cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            cudaMemcpyAsync(c->sc_box_d, sc_box.data(), sizeof(int) * nsc, cudaMemcpyHostToDevice,
                            c->stream) != cudaSuccess ||
            cudaMemcpyAsync(c->items_d, items.data(), sizeof(int) * nsc, cudaMemcpyHostToDevice,
                            c->stream) != cudaSuccess ||
            cudaMemcpyAsync(c->yee_off_d, yee_off.data(), sizeof(int) * (nboxes + 1),
                            cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            cudaGetLastError();
            return bail(PIC_ERR_CUDA);
        }
        const pic_status mst = encode_tile_maps(c);
        if (mst != PIC_OK)
            return bail(mst);
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return bail(PIC_ERR_CUDA);
    }
    *out = c;
    return PIC_OK;
}

pic_status pic_set_background(pic_ctx* c, int32_t box, double rho_bg)
{
    CKS(check_ctx(c));
    if (!valid_box(c, box) || !std::isfinite(rho_bg))
        return fail(c, PIC_ERR_ARG, "bad box or background");
    c->rho_bg[box] = rho_bg;
    return PIC_OK;
}

// ---------------------------------------------------------------- open y

pic_status pic_set_boundary(pic_ctx* c, int32_t box, const pic_boundary* bnd)
{
    CKS(check_ctx(c));
    if (!valid_box(c, box) || !bnd)
        return fail(c, PIC_ERR_ARG, "bad arguments to pic_set_boundary");
    if (c->precision != PIC_PRECISION_MIXED)
        return fail(c, PIC_ERR_ARG, "open y boundaries need the mixed form");
    if (c->sub_z)
        return fail(c, PIC_ERR_ARG, "open-y options do not combine with a subdomain slab");
    BoxDev& b = c->boxes_h[box];
    if (bnd->absorber_cells < 0 || 2 * (int64_t)bnd->absorber_cells > b.ny ||
        !(bnd->absorber_sigma >= 0.0) || !std::isfinite(bnd->absorber_sigma))
        return fail(c, PIC_ERR_ARG, "absorber needs 0 <= 2 cells <= ny and a finite sigma >= 0");
    b.oy.open_y = bnd->open_y != 0;
    b.oy.abs_cells = bnd->absorber_cells;
    b.oy.abs_sigma = (float)bnd->absorber_sigma;
    return upload_boxes(c);
}

pic_status pic_set_antenna(pic_ctx* c, int32_t box, const pic_antenna* a)
{
    CKS(check_ctx(c));
    if (!valid_box(c, box) || !a)
        return fail(c, PIC_ERR_ARG, "bad arguments to pic_set_antenna");
    if (c->precision != PIC_PRECISION_MIXED)
        return fail(c, PIC_ERR_ARG, "the antenna needs the mixed form");
    if (c->sub_z)
        return fail(c, PIC_ERR_ARG, "open-y options do not combine with a subdomain slab");
    BoxDev& b = c->boxes_h[box];
    if (a->plane_y < 0) {
        b.oy.ant_j = -1;
        return upload_boxes(c);
    }
    const double vals[7] = {a->E0, a->omega, a->w0, a->xc, a->zc, a->tau, a->t0};
    for (double v : vals)
        if (!std::isfinite(v))
            return fail(c, PIC_ERR_ARG, "non-finite antenna parameter");
    // Yee dispersion along y: sin(kappa/2) = (dy/dt) sin(omega dt/2)
    const double sk = (c->h[1] / c->dt) * std::sin(0.5 * a->omega * c->dt);
    if (a->plane_y >= b.ny || !(std::fabs(sk) < 1.0))
        return fail(c, PIC_ERR_ARG, "antenna plane outside the box or omega not resolved by the grid");
    const double kappa = 2.0 * std::asin(sk);
    b.oy.ant_j = a->plane_y;
    b.oy.ant_J0 = -2.0 * a->E0 * std::cos(0.5 * kappa) / c->h[1];
    b.oy.ant_omega = a->omega;
    b.oy.ant_w0 = a->w0;
    b.oy.ant_xc = a->xc;
    b.oy.ant_zc = a->zc;
    b.oy.ant_tau = a->tau;
    b.oy.ant_t0 = a->t0;
    return upload_boxes(c);
}

pic_status pic_shift_window(pic_ctx* c, int32_t box, int32_t cells)
{
    CKS(check_ctx(c));
    if (!valid_box(c, box))
        return fail(c, PIC_ERR_ARG, "bad box");
    if (c->precision != PIC_PRECISION_MIXED)
        return fail(c, PIC_ERR_ARG, "the moving window needs the mixed form");
    if (c->sub_z)
        return fail(c, PIC_ERR_ARG, "open-y options do not combine with a subdomain slab");
    const BoxDev& b = c->boxes_h[box];
    if (cells <= 0 || cells >= b.ny || cells % c->LY)
        return fail(c, PIC_ERR_ARG, "shift must be a positive multiple of the supercell edge along y, below ny");
    const int rows = cells / c->LY;
    CK(cudaStreamSynchronize(c->stream));
    // fields: E and B through a copy of the box's field
    const int64_t pf = 3 * padded_cells(b);
    if (c->shift_scratch_floats < pf) {
        raw_free(c, c->shift_scratch);
        c->shift_scratch = nullptr;
        c->shift_scratch_floats = 0;
        CKS(dalloc(c, &c->shift_scratch, pf, false));
        c->shift_scratch_floats = pf;
    }
    for (float* F : {b.E, b.B}) {
        CK(cudaMemcpyAsync(c->shift_scratch, F, sizeof(float) * pf, cudaMemcpyDeviceToDevice, c->stream));
        CK(launch_shift_fields(b, F, c->shift_scratch, cells, c->stream));
    }
    CK(cudaMemsetAsync(b.J, 0, sizeof(float) * pf, c->stream));
    // particles: empty the bottom rows, release their frames through one
    // maintenance pass, then rotate the box's lists down by `rows`
    StepDev d = make_step(c, c->parity);
    d.step_ctr = nullptr;
    CK(launch_clear_rows(d, b, rows, c->stream));
    CK(cudaMemsetAsync(c->mv_count, 0, sizeof(int), c->stream));
    CK(launch_frame_plan(d, c->stream));
    CK(launch_frame_apply(d, 4 * c->nsm, c->stream));
    CKS(status_check(c));
    c->parity ^= 1;
    if (!c->rot_scratch)
        CKS(dalloc(c, &c->rot_scratch, 3 * (int64_t)c->nlists, false));
    CK(cudaMemcpyAsync(c->rot_scratch, c->count, sizeof(int) * c->nlists, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->rot_scratch + c->nlists, c->nframes, sizeof(int) * c->nlists,
                       cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->rot_scratch + 2 * c->nlists, c->foff[c->parity], sizeof(int) * c->nlists,
                       cudaMemcpyDeviceToDevice, c->stream));
    d = make_step(c, c->parity);
    CK(launch_rotate_lists(d, b, c->rot_scratch, c->foff[c->parity], rows, c->stream));
    // a shift by whole supercells keeps every particle's cell and its list
    // order: nothing else to redo
    CK(cudaStreamSynchronize(c->stream));
    return status_check(c);
}

pic_status pic_load_particles(pic_ctx* c, int32_t box, int32_t species, int64_t n,
                              const double* x, const double* u, const double* w)
{
    CKS(check_ctx(c));
    if (!valid_box(c, box) || species < 0 || species >= (int)c->sp.size() || n < 0 ||
        (n > 0 && (!x || !u)))
        return fail(c, PIC_ERR_ARG, "bad arguments to pic_load_particles");
    if (n == 0)
        return PIC_OK;
    int64_t& idn = c->id_next[(size_t)box * c->sp.size() + species];
    if (idn + n > INT32_MAX)
        return fail(c, PIC_ERR_ARG, "more than 2^31 particles in one (box, species)");
    // captured step graphs stay valid unless a buffer they use is reallocated
    // (ensure_pool / ensure_mv drop them) or a weight bound grows (below)
    const int64_t chunk = std::min<int64_t>(n, 1 << 25);  // 32 M particles: 1.9 GB of FP64 staging
    // mixed form from page-locked host arrays: the conversion reads them in place
    const double* hx = nullptr;
    const double* hu = nullptr;
    const double* hw = nullptr;
    if (c->precision != PIC_PRECISION_FP64_PLAIN) {
        hx = static_cast<const double*>(host_range_on_device(x, sizeof(double) * 3 * (size_t)n));
        hu = static_cast<const double*>(host_range_on_device(u, sizeof(double) * 3 * (size_t)n));
        hw = w ? static_cast<const double*>(host_range_on_device(w, sizeof(double) * (size_t)n)) : nullptr;
    }
    const bool direct = hx && hu && (!w || hw);
    if (direct)
        ++c->host_direct;
    else
        CKS(ensure_stage(c, sizeof(double) * 7 * (size_t)chunk));
    if (c->precision != PIC_PRECISION_FP64_PLAIN) {
        // one pool growth for the whole call instead of one per chunk (each
        // growth reallocates and copies every pool array): room for what the
        // call can add -- every particle, plus one part-filled frame per list
        // of the box -- and for the first step's headroom (prepare_mixed), so
        // that the first step does not grow the pool either.  A capacity set
        // in the options is taken as given (the chunks below still add what
        // an insertion needs beyond it).
        if (c->opt.pool_frames > 0) {
            CKS(ensure_pool(c, c->opt.pool_frames));
        } else {
            int top = 0;
            if (c->pool_cap > 0)
                CKS(read_free_top(c, &top));
            const BoxDev& bd = c->boxes_h[box];
            const int64_t lists = (int64_t)bd.nscx * bd.nscy * bd.nscz;
            const int64_t after = (c->pool_cap - top) + (n + c->S - 1) / c->S + std::min<int64_t>(n, lists);
            CKS(ensure_pool(c, after + after / 4 + c->nlists / 4 + 1024));
        }
    }
    for (int64_t b0 = 0; b0 < n; b0 += chunk) {
        const int64_t m = std::min(chunk, n - b0);
        const double *sx, *su, *sw;
        if (direct) {
            sx = hx + 3 * b0;
            su = hu + 3 * b0;
            sw = w ? hw + b0 : nullptr;
        } else {
            double* st = static_cast<double*>(c->stage_d);
            CK(cudaMemcpyAsync(st, x + 3 * b0, sizeof(double) * 3 * m, cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemcpyAsync(st + 3 * chunk, u + 3 * b0, sizeof(double) * 3 * m, cudaMemcpyHostToDevice,
                               c->stream));
            if (w)
                CK(cudaMemcpyAsync(st + 6 * chunk, w + b0, sizeof(double) * m, cudaMemcpyHostToDevice,
                                   c->stream));
            sx = st;
            su = st + 3 * chunk;
            sw = w ? st + 6 * chunk : nullptr;
        }
        if (c->precision == PIC_PRECISION_FP64_PLAIN) {
            PlainSpecies& s = c->pboxes[box].sp[species];
            CKS(plain_grow(c, s, s.n + m));
            const pic_grid& g = c->grids[box];
            CK(launch_plain_load(m, sx, su, sw, g.nx, g.ny, g.nz, s.x + s.n, s.y + s.n,
                                 s.z + s.n, s.ux + s.n, s.uy + s.n, s.uz + s.n, s.w + s.n,
                                 s.pid ? s.pid + s.n : nullptr, (int)(idn + b0), c->status_d,
                                 c->stream));
            unsigned st = 0;
            CK(cudaMemcpyAsync(&st, c->status_d, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            if (st) {
                CK(cudaMemsetAsync(c->status_d, 0, sizeof(unsigned), c->stream));
                CK(cudaStreamSynchronize(c->stream));
                return fail(c, PIC_ERR_ARG, "non-finite particle data");
            }
            s.n += m;
        } else {
            CKS(insert_mixed(c, box, species, m, sx, su, sw, (int)(idn + b0), nullptr));
        }
    }
    idn += n;
    c->total_particles += n;
    c->prepared = false;
    return PIC_OK;
}

}  // extern "C"

namespace {

// Mixed form: convert m particles from device (or mapped host) FP64 arrays
// into box `box`'s frame lists (ids: per particle, or null for id_base + i).
pic_status insert_mixed(pic_ctx* c, int box, int species, int64_t m, const double* sx, const double* su,
                        const double* sw, int id_base, const int64_t* ids)
{
    {
        {
            CKS(ensure_mv(c, std::max<int64_t>(c->mv_cap, m)));
            StepDev d = make_step(c, c->parity);
            CK(launch_insert_convert(d, box, species, m, sx, su, sw, id_base, ids, c->stream));
            int mi = (int)m;
            CK(cudaMemcpyAsync(c->mv_count, &mi, sizeof(int), cudaMemcpyHostToDevice, c->stream));
            unsigned st = 0;
            unsigned wbits[kMaxSpecies];
            CK(cudaMemcpyAsync(&st, c->status_d, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaMemcpyAsync(wbits, c->wmax_bits, sizeof(wbits), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            float wm;
            std::memcpy(&wm, &wbits[species], sizeof(float));
            if (wm > c->wmax[species]) {
                c->wmax[species] = wm;  // the push kernels bake the bound in: recapture
                destroy_graphs(c);
            }
            if (st) {
                CK(cudaMemsetAsync(c->narrive, 0, sizeof(int) * c->nlists, c->stream));
                CK(cudaMemsetAsync(c->status_d, 0, sizeof(unsigned), c->stream));
                CK(cudaMemsetAsync(c->mv_count, 0, sizeof(int), c->stream));
                CK(cudaStreamSynchronize(c->stream));
                return fail(c, PIC_ERR_ARG, "non-finite particle data");
            }
            // count the frames this insertion needs, grow the pool, then place;
            // the next step is a sort pass (the arrivals sit unsorted at the
            // list ends)
            d.step_ctr = nullptr;
            CK(cudaMemsetAsync(c->step_ctr, 0, sizeof(int), c->stream));
            CK(launch_frame_plan(d, c->stream));
            int4 tot;
            int top = 0;
            CK(cudaMemcpyAsync(&tot, c->totals, sizeof(int4), cudaMemcpyDeviceToHost, c->stream));
            CKS(read_free_top(c, &top));
            if (tot.y > top)
                CKS(ensure_pool(c, (c->pool_cap - top) + tot.y));
            d = make_step(c, c->parity);
            CK(launch_frame_apply(d, 4 * c->nsm, c->stream));
            CKS(status_check(c));
            c->parity ^= 1;
        }
    }
    return PIC_OK;
}

}  // namespace

extern "C" {

pic_status pic_write_fields(pic_ctx* c, int32_t box, int32_t which, const double* f)
{
    CKS(check_ctx(c));
    if (!valid_box(c, box) || (which != PIC_FIELD_E && which != PIC_FIELD_B) || !f)
        return fail(c, PIC_ERR_ARG, "bad arguments to pic_write_fields");
    const pic_grid& g = c->grids[box];
    const int64_t nc = (int64_t)g.nx * g.ny * g.nz;
    if (c->precision == PIC_PRECISION_FP64_PLAIN) {
        double* dst = which == PIC_FIELD_E ? c->pboxes[box].E : c->pboxes[box].B;
        CK(cudaMemcpyAsync(dst, f, sizeof(double) * 3 * nc, cudaMemcpyHostToDevice, c->stream));
    } else {
        CKS(ensure_stage(c, sizeof(double) * 3 * nc));
        CK(cudaMemcpyAsync(c->stage_d, f, sizeof(double) * 3 * nc, cudaMemcpyHostToDevice, c->stream));
        CK(launch_fields_to_padded(c->boxes_h[box], which, static_cast<double*>(c->stage_d),
                                   c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

pic_status pic_step_async(pic_ctx* c, int32_t nsteps)
{
    CKS(check_ctx(c));
    if (nsteps < 0)
        return fail(c, PIC_ERR_ARG, "nsteps < 0");
    if (c->precision == PIC_PRECISION_FP64_PLAIN) {
        for (int i = 0; i < nsteps; ++i) {
            cudaEvent_t* ev = nullptr;
            if (c->timing)
                CKS(step_events(c, &ev));
            CKS(enqueue_step_plain(c, ev));
            ++c->steps_done;
        }
        return PIC_OK;
    }
    if (c->sub_z)
        return fail(c, PIC_ERR_ARG, "a subdomain context steps through pic_step_stage");
    if (c->next_stage != PIC_STAGE_PUSH)
        return fail(c, PIC_ERR_ARG, "a step begun with pic_step_stage is not finished");
    if (c->tune_pending && nsteps > 0)
        CKS(autotune(c));
    CKS(prepare_mixed(c));
    if (c->opt.use_graph) {
        CKS(capture_graphs(c));
        if (nsteps >= 2)
            CKS(capture_pair_graphs(c));
    }
    for (int i = 0; i < nsteps;) {
        cudaEvent_t* ev = nullptr;
        if (c->fused_ready && nsteps - i >= 2) {
            // a pair with the fused field update: the fields go to the
            // second buffer pair and back
            if (c->timing)
                CKS(step_events(c, &ev, 2));
            if (c->opt.use_graph && c->pgexec[c->parity])
                CKS(launch_pair_graph(c, c->parity, ev));
            else
                CKS(enqueue_pair_mixed(c, c->parity, ev));
            c->steps_done += 2;
            c->fused_steps += 2;
            i += 2;
            continue;
        }
        if (c->timing)
            CKS(step_events(c, &ev));
        if (c->opt.use_graph && c->gexec[c->parity])
            CKS(launch_graph(c, c->parity, ev));
        else
            CKS(enqueue_step_mixed(c, c->parity, ev));
        c->parity ^= 1;
        ++c->steps_done;
        ++i;
    }
    return PIC_OK;
}

pic_status pic_sync(pic_ctx* c)
{
    CKS(check_ctx(c));
    return status_check(c);
}

pic_status pic_step(pic_ctx* c, int32_t nsteps)
{
    CKS(pic_step_async(c, nsteps));
    return pic_sync(c);
}

pic_status pic_count_particles(pic_ctx* c, int32_t box, int32_t species, int64_t* n_out)
{
    CKS(check_ctx(c));
    if (!valid_box(c, box) || species < 0 || species >= (int)c->sp.size() || !n_out)
        return fail(c, PIC_ERR_ARG, "bad arguments to pic_count_particles");
    if (c->precision == PIC_PRECISION_FP64_PLAIN) {
        *n_out = c->pboxes[box].sp[species].n;
        return PIC_OK;
    }
    const BoxDev& b = c->boxes_h[box];
    const int nscb = b.nscx * b.nscy * b.nscz;
    std::vector<int> cnt(nscb);
    CK(cudaMemcpyAsync(cnt.data(), c->count + (size_t)species * c->nsc + b.sc_base, sizeof(int) * nscb,
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    int64_t t = 0;
    for (int v : cnt)
        t += v;
    *n_out = t;
    return PIC_OK;
}

}  // extern "C"

namespace {

// Mixed form: convert the (box, species) particles to FP64 into the device
// addresses dx, du, dw, di (each may be null); when a host destination hx..hi
// is given, copy the converted array there afterwards.
pic_status read_particles_mixed(pic_ctx* c, int box, int species, double* dx, double* du, double* dw,
                                int64_t* di, double* hx, double* hu, double* hw, int64_t* hi)
{
    const BoxDev& b = c->boxes_h[box];
    const int nscb = b.nscx * b.nscy * b.nscz;
    std::vector<int> cnt(nscb), off(nscb);
    CK(cudaMemcpyAsync(cnt.data(), c->count + (size_t)species * c->nsc + b.sc_base, sizeof(int) * nscb,
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    int64_t acc = 0;
    for (int i = 0; i < nscb; ++i) {
        off[i] = (int)acc;
        acc += cnt[i];
    }
    const int64_t n = acc;
    CKS(ensure_ioff(c, nscb));
    CK(cudaMemcpyAsync(c->ioff_d, off.data(), sizeof(int) * nscb, cudaMemcpyHostToDevice, c->stream));
    StepDev d = make_step(c, c->parity);
    CK(launch_read_particles(d, b, box, species, c->ioff_d, dx, du, dw, di, c->stream));
    if (hx)
        CK(cudaMemcpyAsync(hx, dx, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
    if (hu)
        CK(cudaMemcpyAsync(hu, du, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
    if (hw)
        CK(cudaMemcpyAsync(hw, dw, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    if (hi)
        CK(cudaMemcpyAsync(hi, di, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

// ------------------------------------------------------------ in-library autotuning

struct TuneCfg {
    int sc[3];
    int threads;
};

// Supercell shapes and thread counts the push kernel is built for that fit
// this context: every box a whole number of supercells, the shared memory
// within the device's limit; only thread counts when the supercell was given.
std::vector<TuneCfg> tune_candidates(const pic_ctx* c)
{
    std::vector<TuneCfg> out;
    const int edges[2] = {4, 8}, threads[3] = {64, 128, 256};
    for (int ez : edges)
        for (int ey : edges)
            for (int ex : edges)
                for (int t : threads) {
                    if (!c->tune_sc && (ex != c->LX || ey != c->LY || ez != c->LZ))
                        continue;
                    if (!c->tune_threads && t != c->threads)
                        continue;
                    if (!push_supported(ex, ey, ez, t, c->guard) ||
                        push_smem_bytes(ex, ey, ez, t, c->guard) > c->smem_optin)
                        continue;
                    bool fits = true;
                    for (const pic_grid& g : c->grids)
                        fits = fits && g.nx % ex == 0 && g.ny % ey == 0 && g.nz % ez == 0;
                    if (fits)
                        out.push_back(TuneCfg{{ex, ey, ez}, t});
                }
    return out;
}

// What the result of a tuning depends on: box sizes, species, guard,
// particles per cell (to 0.5), and which of the two was left to the tuner.
std::string tune_key(const pic_ctx* c)
{
    std::string k;
    char buf[160];
    int64_t cells = 0;
    for (const pic_grid& g : c->grids) {
        snprintf(buf, sizeof(buf), "%d,%d,%d;", g.nx, g.ny, g.nz);
        k += buf;
        cells += (int64_t)g.nx * g.ny * g.nz;
    }
    for (const pic_species& p : c->sp) {
        snprintf(buf, sizeof(buf), "%.17g,%.17g,%d,%d,%d;", p.charge, p.mass, p.shape, p.mobile, p.gather);
        k += buf;
    }
    const double ppc = cells > 0 ? (double)c->total_particles / (double)cells : 0.0;
    snprintf(buf, sizeof(buf), "g%d|ppc%.1f|%d%d|%d", c->guard, std::round(2.0 * ppc) / 2.0, (int)c->tune_sc,
             (int)c->tune_threads, c->sort_every);
    return k + buf;
}

std::mutex g_tune_mutex;
std::map<std::string, TuneCfg> g_tune_cache;  // per process

// The particles (FP64 global form, ids when tracked) and the E, B arrays of
// a context, in device buffers from its allocator.
struct TuneSnapshot {
    struct Part {
        int box, species;
        int64_t n;
        double *x, *u, *w;
        int64_t* id;
    };
    std::vector<Part> parts;
    float *E = nullptr, *B = nullptr;
};

pic_status take_snapshot(pic_ctx* c, TuneSnapshot* snap)
{
    for (int b = 0; b < c->nboxes; ++b)
        for (int s = 0; s < (int)c->sp.size(); ++s) {
            int64_t n = 0;
            CKS(pic_count_particles(c, b, s, &n));
            TuneSnapshot::Part p{b, s, n, nullptr, nullptr, nullptr, nullptr};
            if (n > 0) {
                CKS(dalloc(c, &p.x, 3 * n, false));
                CKS(dalloc(c, &p.u, 3 * n, false));
                CKS(dalloc(c, &p.w, n, false));
                if (c->opt.track_ids)
                    CKS(dalloc(c, &p.id, n, false));
                CKS(read_particles_mixed(c, b, s, p.x, p.u, p.w, p.id, nullptr, nullptr, nullptr, nullptr));
            }
            snap->parts.push_back(p);
        }
    CKS(dalloc(c, &snap->E, c->field_floats, false));
    CKS(dalloc(c, &snap->B, c->field_floats, false));
    CK(cudaMemcpyAsync(snap->E, c->E_all, sizeof(float) * c->field_floats, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(snap->B, c->B_all, sizeof(float) * c->field_floats, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

void drop_snapshot(pic_ctx* c, TuneSnapshot* snap)
{
    for (auto& p : snap->parts) {
        raw_free(c, p.x);
        raw_free(c, p.u);
        raw_free(c, p.w);
        raw_free(c, p.id);
    }
    raw_free(c, snap->E);
    raw_free(c, snap->B);
    snap->parts.clear();
}

// A context like c (grids, cell, time step, species, options, stream,
// allocator, boundaries, backgrounds, ids) in configuration cfg, holding the
// snapshot's particles and fields.
pic_status build_like(pic_ctx* c, const TuneCfg& cfg, const TuneSnapshot& snap, pic_ctx** out)
{
    pic_options o = c->opt;
    o.sc[0] = cfg.sc[0];
    o.sc[1] = cfg.sc[1];
    o.sc[2] = cfg.sc[2];
    o.threads_per_sc = cfg.threads;
    o.stream = c->stream;
    pic_ctx* n = nullptr;
    pic_status st = pic_create(c->grids.data(), c->nboxes, c->h, c->dt, c->sp.data(), (int)c->sp.size(), &o, &n);
    if (st != PIC_OK)
        return st;
    auto bail = [&](pic_status e) {
        pic_destroy(n);
        return e;
    };
    n->rho_bg = c->rho_bg;
    for (int b = 0; b < c->nboxes; ++b)
        n->boxes_h[b].oy = c->boxes_h[b].oy;
    if ((st = upload_boxes(n)) != PIC_OK)
        return bail(st);
    // one pool growth for all insertions: every particle, one part-filled
    // frame per list, and the first step's headroom
    int64_t frames = 0;
    for (const auto& p : snap.parts)
        frames += (p.n + n->S - 1) / n->S;
    frames += n->nlists;
    if ((st = ensure_pool(n, frames + frames / 4 + 1024)) != PIC_OK)
        return bail(st);
    for (const auto& p : snap.parts) {
        if (p.n == 0)
            continue;
        if ((st = insert_mixed(n, p.box, p.species, p.n, p.x, p.u, p.w, 0, p.id)) != PIC_OK)
            return bail(st);
        n->total_particles += p.n;
    }
    n->id_next = c->id_next;
    if (cudaMemcpyAsync(n->E_all, snap.E, sizeof(float) * c->field_floats, cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess ||
        cudaMemcpyAsync(n->B_all, snap.B, sizeof(float) * c->field_floats, cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return bail(PIC_ERR_CUDA);
    }
    *out = n;
    return PIC_OK;
}

// Push + frame maintenance milliseconds per step of configuration cfg on
// the snapshot: after one warm-up step (the sort pass that follows a load),
// two whole sort periods timed with the step's stage events, so that sort
// and stored-order passes weigh as they do in a run.
double time_config(pic_ctx* c, const TuneCfg& cfg, const TuneSnapshot& snap)
{
    pic_ctx* n = nullptr;
    if (build_like(c, cfg, snap, &n) != PIC_OK)
        return INFINITY;
    double ms[4] = {0, 0, 0, 0};
    int64_t k = 0;
    const bool ok = pic_step(n, 1) == PIC_OK && pic_stage_timing(n, 1) == PIC_OK &&
                    pic_step(n, 2 * n->sort_every) == PIC_OK && pic_stage_times(n, ms, &k) == PIC_OK && k > 0;
    pic_destroy(n);
    cudaGetLastError();
    return ok ? (ms[0] + ms[1]) / (double)k : INFINITY;
}

// Before the first step of a context created with sc = 0,0,0 and/or
// threads_per_sc = 0: time every candidate on the loaded state (or take the
// result of an earlier tuning of the same kind of state in this process),
// then move the context into the fastest configuration.  The context's
// state (particles with their ids, fields, backgrounds, boundaries) is the
// same afterwards; only its supercells and threads change.
pic_status autotune(pic_ctx* c)
{
    c->tune_pending = false;
    if (c->total_particles == 0 || c->steps_done != 0)
        return PIC_OK;
    const std::vector<TuneCfg> cands = tune_candidates(c);
    if (cands.empty())
        return PIC_OK;
    const std::string key = tune_key(c);
    TuneCfg best = cands[0];
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best = it->second;
            cached = true;
        }
    }
    TuneSnapshot snap;
    pic_status st = take_snapshot(c, &snap);
    if (st != PIC_OK) {
        drop_snapshot(c, &snap);
        return st;
    }
    if (!cached) {
        double best_ms = INFINITY;
        for (const TuneCfg& cfg : cands) {
            const double ms = time_config(c, cfg, snap);
            if (ms < best_ms) {
                best_ms = ms;
                best = cfg;
            }
        }
        c->tune_trials = (int)cands.size();
        if (!(best_ms < INFINITY)) {  // no candidate ran: keep the configuration in use
            drop_snapshot(c, &snap);
            return PIC_OK;
        }
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = best;
    } else {
        c->tune_trials = 0;
    }
    if (best.sc[0] == c->LX && best.sc[1] == c->LY && best.sc[2] == c->LZ && best.threads == c->threads) {
        drop_snapshot(c, &snap);
        return PIC_OK;
    }
    pic_ctx* n = nullptr;
    st = build_like(c, best, snap, &n);
    drop_snapshot(c, &snap);
    if (st != PIC_OK)
        return fail(c, st, "autotune: rebuilding the context in supercell %dx%dx%d, %d threads failed",
                    best.sc[0], best.sc[1], best.sc[2], best.threads);
    // c takes n's state; n takes c's old state and releases it
    const bool own = c->own_stream, timing = c->timing;
    const pic_options user = c->opt;
    const int trials = c->tune_trials;
    const int64_t host_direct = c->host_direct;
    std::swap(*c, *n);
    c->own_stream = own;
    n->own_stream = false;
    c->opt = user;
    c->tune_trials = trials;
    c->host_direct = host_direct;
    c->timing = timing;
    c->tune_sc = n->tune_sc;
    c->tune_threads = n->tune_threads;
    pic_destroy(n);
    return PIC_OK;
}

}  // namespace

extern "C" {

pic_status pic_read_particles(pic_ctx* c, int32_t box, int32_t species, int64_t cap, double* x,
                              double* u, double* w, int64_t* id, int64_t* n_out)
{
    CKS(check_ctx(c));
    if (!valid_box(c, box) || species < 0 || species >= (int)c->sp.size() || !n_out || cap < 0)
        return fail(c, PIC_ERR_ARG, "bad arguments to pic_read_particles");
    if (id && !c->opt.track_ids)
        return fail(c, PIC_ERR_ARG, "particle ids requested but track_ids is off");
    CK(cudaStreamSynchronize(c->stream));
    int64_t n = 0;
    CKS(pic_count_particles(c, box, species, &n));
    *n_out = n;
    if (n > cap)
        return fail(c, PIC_ERR_ARG, "cap %lld below the particle count %lld", (long long)cap,
                    (long long)n);
    if (n == 0)
        return PIC_OK;
    // mixed form into page-locked host arrays: the conversion writes them in place
    if (c->precision != PIC_PRECISION_FP64_PLAIN) {
        void* dx = x ? const_cast<void*>(host_range_on_device(x, sizeof(double) * 3 * (size_t)n)) : nullptr;
        void* du = u ? const_cast<void*>(host_range_on_device(u, sizeof(double) * 3 * (size_t)n)) : nullptr;
        void* dw = w ? const_cast<void*>(host_range_on_device(w, sizeof(double) * (size_t)n)) : nullptr;
        void* di = id ? const_cast<void*>(host_range_on_device(id, sizeof(int64_t) * (size_t)n)) : nullptr;
        if ((!x || dx) && (!u || du) && (!w || dw) && (!id || di)) {
            ++c->host_direct;
            return read_particles_mixed(c, box, species, static_cast<double*>(dx), static_cast<double*>(du),
                                        static_cast<double*>(dw), static_cast<int64_t*>(di), nullptr, nullptr,
                                        nullptr, nullptr);
        }
    }
    CKS(ensure_stage(c, sizeof(double) * 7 * (size_t)n + sizeof(int64_t) * (size_t)n));
    double* sx = static_cast<double*>(c->stage_d);
    double* su = sx + 3 * n;
    double* sw = su + 3 * n;
    int64_t* sid = reinterpret_cast<int64_t*>(sw + n);
    if (c->precision == PIC_PRECISION_FP64_PLAIN) {
        PlainSpecies& s = c->pboxes[box].sp[species];
        CK(launch_plain_interleave(n, s.x, s.y, s.z, sx, c->stream));
        CK(launch_plain_interleave(n, s.ux, s.uy, s.uz, su, c->stream));
        if (x)
            CK(cudaMemcpyAsync(x, sx, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
        if (u)
            CK(cudaMemcpyAsync(u, su, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
        if (w)
            CK(cudaMemcpyAsync(w, s.w, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
        if (id) {
            std::vector<int> tmp((size_t)n);
            CK(cudaMemcpyAsync(tmp.data(), s.pid, sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            for (int64_t i = 0; i < n; ++i)
                id[i] = tmp[(size_t)i];
        }
        CK(cudaStreamSynchronize(c->stream));
        return PIC_OK;
    }
    return read_particles_mixed(c, box, species, sx, su, sw, id ? sid : nullptr, x, u, w, id);
}

pic_status pic_diagnostics(pic_ctx* c, int32_t box, double out[4])
{
    CKS(check_ctx(c));
    if (!valid_box(c, box) || !out)
        return fail(c, PIC_ERR_ARG, "bad arguments to pic_diagnostics");
    const double vol = c->h[0] * c->h[1] * c->h[2];
    const pic_grid& g = c->grids[box];
    const int64_t nc = (int64_t)g.nx * g.ny * g.nz;
    if (c->precision == PIC_PRECISION_FP64_PLAIN) {
        CK(cudaMemsetAsync(c->rho_d, 0, sizeof(double) * nc, c->stream));
        CK(cudaMemsetAsync(c->diag_d, 0, sizeof(double) * 4, c->stream));
        PlainYeeArgs ya = plain_yee_args(c, box);
        CK(launch_plain_diag_fields(ya, c->diag_d, vol, c->stream));
        for (size_t s = 0; s < c->sp.size(); ++s)
            CK(launch_plain_diag_particles(plain_args(c, box, (int)s), c->sp[s].shape, c->sp[s].mass,
                                           c->sp[s].charge, 1.0 / vol, c->rho_d, c->diag_d, c->stream));
        CK(launch_plain_diag_gauss(ya, c->rho_d, c->rho_bg[box], c->diag_d, c->stream));
    } else {
        StepDev d = make_step(c, c->parity);
        CK(launch_diag_mixed(d, c->boxes_h[box], box, c->rho_bg[box], c->rho_d, c->diag_d, c->h,
                             c->stream));
    }
    CK(cudaMemcpyAsync(out, c->diag_d, sizeof(double) * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    out[2] += c->rho_bg[box] * vol * (double)nc;
    return PIC_OK;
}

pic_status pic_read_fields(pic_ctx* c, int32_t box, int32_t which, double* out)
{
    CKS(check_ctx(c));
    if (!valid_box(c, box) || which < PIC_FIELD_E || which > PIC_FIELD_RHO || !out)
        return fail(c, PIC_ERR_ARG, "bad arguments to pic_read_fields");
    const pic_grid& g = c->grids[box];
    const int64_t nc = (int64_t)g.nx * g.ny * g.nz;
    if (which == PIC_FIELD_RHO) {
        double tmp[4];
        CKS(pic_diagnostics(c, box, tmp));
        CK(cudaMemcpyAsync(out, c->rho_d, sizeof(double) * nc, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (int64_t i = 0; i < nc; ++i)
            out[i] += c->rho_bg[box];
        return PIC_OK;
    }
    if (c->precision == PIC_PRECISION_FP64_PLAIN) {
        const PlainBox& b = c->pboxes[box];
        const double* src = which == PIC_FIELD_E ? b.E : (which == PIC_FIELD_B ? b.B : b.J);
        CK(cudaMemcpyAsync(out, src, sizeof(double) * 3 * nc, cudaMemcpyDeviceToHost, c->stream));
    } else if (void* dout = const_cast<void*>(host_range_on_device(out, sizeof(double) * 3 * nc))) {
        // page-locked destination: the conversion writes it in place
        ++c->host_direct;
        CK(launch_fields_from_padded(c->boxes_h[box], which, static_cast<double*>(dout), c->stream));
    } else {
        CKS(ensure_stage(c, sizeof(double) * 3 * nc));
        CK(launch_fields_from_padded(c->boxes_h[box], which, static_cast<double*>(c->stage_d),
                                     c->stream));
        CK(cudaMemcpyAsync(out, c->stage_d, sizeof(double) * 3 * nc, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

pic_status pic_stage_timing(pic_ctx* c, int32_t enable)
{
    CKS(check_ctx(c));
    CKS(harvest_events(c));
    c->timing = enable != 0;
    for (double& v : c->acc_ms)
        v = 0.0;
    c->timed_steps = 0;
    return PIC_OK;
}

pic_status pic_stage_times(pic_ctx* c, double ms[4], int64_t* nsteps_out)
{
    CKS(check_ctx(c));
    if (!ms)
        return fail(c, PIC_ERR_ARG, "ms is NULL");
    CKS(harvest_events(c));
    for (int i = 0; i < kStageTimers; ++i)
        ms[i] = c->acc_ms[i];
    if (nsteps_out)
        *nsteps_out = c->timed_steps;
    return PIC_OK;
}

pic_status pic_info(pic_ctx* c, int32_t key, int64_t* out)
{
    CKS(check_ctx(c));
    if (!out)
        return fail(c, PIC_ERR_ARG, "out is NULL");
    switch (key) {
    case PIC_INFO_GRAPH_ACTIVE:
        *out = (c->precision == PIC_PRECISION_MIXED && c->gexec[0] && c->gexec[1]) ? 1 : 0;
        return PIC_OK;
    case PIC_INFO_KERNELS_PER_STEP:
        if (c->precision == PIC_PRECISION_MIXED) {
            // push; scan reduce, top; apply, place, free; Yee x3; antenna; y absorber;
            // a subdomain slab adds its 16 halo pack/unpack launches (J, B, E, B:
            // two faces each way) and 2 migrant accepts
            // (the fused field update: one kernel for the three)
            const bool fused = c->fused_ready;
            *out = 1 + 2 + 3 + (fused ? 1 : 3) + (c->any_antenna ? 1 : 0) + (c->abs_nblocks > 0 ? 1 : 0) +
                   (c->sub_z ? 18 : 0);
        } else {
            int64_t k = 0;
            for (int b = 0; b < c->nboxes; ++b) {
                for (size_t s = 0; s < c->sp.size(); ++s)
                    k += (c->sp[s].mobile && c->pboxes[b].sp[s].n > 0) ? 1 : 0;
                k += 3;
            }
            *out = k;
        }
        return PIC_OK;
    case PIC_INFO_POOL_FRAMES:
        *out = c->pool_cap;
        return PIC_OK;
    case PIC_INFO_FRAMES_USED: {
        if (c->precision != PIC_PRECISION_MIXED || c->pool_cap == 0) {
            *out = 0;
            return PIC_OK;
        }
        int top = 0;
        CKS(read_free_top(c, &top));
        *out = c->pool_cap - top;
        return PIC_OK;
    }
    case PIC_INFO_STEPS:
        *out = c->steps_done;
        return PIC_OK;
    case PIC_INFO_FUSED_STEPS:
        *out = c->fused_steps;
        return PIC_OK;
    case PIC_INFO_FIELD_UPDATE:
        *out = c->fused_ready ? PIC_FIELD_UPDATE_FUSED
                              : (c->field_chosen || c->opt.field_update == PIC_FIELD_UPDATE_IN_PLACE || c->sub_z
                                     ? PIC_FIELD_UPDATE_IN_PLACE
                                     : PIC_FIELD_UPDATE_AUTO);
        return PIC_OK;
    case PIC_INFO_HOST_DIRECT:
        *out = c->host_direct;
        return PIC_OK;
    case PIC_INFO_MOVE_CAPACITY:
        *out = c->mv_cap;
        return PIC_OK;
    case PIC_INFO_SUPERCELL_X:
    case PIC_INFO_SUPERCELL_Y:
    case PIC_INFO_SUPERCELL_Z:
        *out = c->precision == PIC_PRECISION_MIXED
                   ? (key == PIC_INFO_SUPERCELL_X ? c->LX : (key == PIC_INFO_SUPERCELL_Y ? c->LY : c->LZ))
                   : 0;
        return PIC_OK;
    case PIC_INFO_THREADS:
        *out = c->precision == PIC_PRECISION_MIXED ? c->threads : 0;
        return PIC_OK;
    case PIC_INFO_TUNE_TRIALS:
        *out = c->tune_trials;
        return PIC_OK;
    default:
        return fail(c, PIC_ERR_ARG, "unknown info key %d", key);
    }
}

// ------------------------------------------------------------ domain decomposition (z slabs)

pic_status pic_set_subdomain(pic_ctx* c, int32_t box, const pic_subdomain* sub)
{
    CKS(check_ctx(c));
    if (!sub || box != 0 || c->nboxes != 1)
        return fail(c, PIC_ERR_ARG, "a subdomain is box 0 of a one-box context");
    if (c->precision != PIC_PRECISION_MIXED)
        return fail(c, PIC_ERR_ARG, "subdomains need the mixed form");
    if (c->next_stage != PIC_STAGE_PUSH)
        return fail(c, PIC_ERR_ARG, "pic_set_subdomain in the middle of a step");
    BoxDev& b = c->boxes_h[0];
    if (b.oy.open_y || b.oy.abs_cells > 0 || b.oy.ant_j >= 0)
        return fail(c, PIC_ERR_ARG, "open-y options do not combine with a subdomain slab");
    if (sub->migrant_capacity < 0 || sub->migrant_capacity > (1 << 26))
        return fail(c, PIC_ERR_ARG, "migrant_capacity out of range");
    if (sub->id_base < 0 || sub->id_base > INT32_MAX)
        return fail(c, PIC_ERR_ARG, "id_base out of range");
    if (sub->enable) {
        const int64_t cap = sub->migrant_capacity > 0 ? sub->migrant_capacity : 2 * (int64_t)b.nx * b.ny;
        if (cap != c->mig_cap) {
            CK(cudaStreamSynchronize(c->stream));
            raw_free(c, c->mig);
            c->mig = nullptr;
            const int64_t bytes = (int64_t)sizeof(MigHeader) + cap * (int64_t)sizeof(MigRec);
            CKS(dalloc(c, &c->mig, 2 * bytes, true));
            const MigHeader h{0, (int)cap, {0, 0}};
            CK(cudaMemcpyAsync(c->mig, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemcpyAsync(c->mig + bytes, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
            c->mig_bytes = bytes;
            c->mig_cap = (int)cap;
        }
    }
    b.sub_z = sub->enable ? 1 : 0;
    c->sub_z = sub->enable != 0;
    if (c->sub_z)
        c->tune_pending = false;  // slabs keep the configuration they were created with
    if (sub->enable)
        for (auto& v : c->id_next)
            v = sub->id_base;
    destroy_graphs(c);
    return upload_boxes(c);
}

pic_status pic_step_stage(pic_ctx* c, int32_t stage)
{
    CKS(check_ctx(c));
    if (c->precision != PIC_PRECISION_MIXED)
        return fail(c, PIC_ERR_ARG, "pic_step_stage needs the mixed form");
    if (stage != c->next_stage)
        return fail(c, PIC_ERR_ARG, "stage %d out of order (expected %d)", stage, c->next_stage);
    if (stage == PIC_STAGE_PUSH)
        CKS(prepare_mixed(c));
    CKS(enqueue_stage(c, stage, c->parity));
    if (stage == PIC_STAGE_FRAMES) {
        c->parity ^= 1;
        ++c->steps_done;
    }
    c->next_stage = (stage + 1) % (PIC_STAGE_B_SECOND + 1);
    return PIC_OK;
}

}  // extern "C"

namespace {

// Padded z planes [p0, p0 + np) of a subdomain box's halo message or its
// target: pack = the message to the neighbour on `side`, else the planes the
// message from the neighbour on `side` goes into.  E, B: interior planes the
// neighbour keeps as guards / this slab's guards; J: this slab's guards /
// its interior planes on that face.
void halo_planes(const BoxDev& b, int which, int side, bool pack, int* p0, int* np)
{
    const int G = b.gz, top = b.pz - b.gz - b.nz;  // guard planes below / above
    const bool j = which == PIC_FIELD_J;
    if (j == pack) {  // E/B unpack or J pack: the guard planes of that face
        *p0 = side == 0 ? 0 : G + b.nz;
        *np = side == 0 ? G : top;
    } else {          // E/B pack or J unpack: the interior planes of that face
        *p0 = side == 0 ? G : b.nz;
        *np = side == 0 ? top : G;
    }
}

pic_status halo_check(pic_ctx* c, int box, int which, int side)
{
    CKS(check_ctx(c));
    if (!c->sub_z || box != 0)
        return fail(c, PIC_ERR_ARG, "halos belong to a subdomain box (pic_set_subdomain)");
    if ((which != PIC_FIELD_E && which != PIC_FIELD_B && which != PIC_FIELD_J) || (side != 0 && side != 1))
        return fail(c, PIC_ERR_ARG, "bad field or side");
    return PIC_OK;
}

float* field_of(pic_ctx* c, int which)
{
    const BoxDev& b = c->boxes_h[0];
    return which == PIC_FIELD_E ? b.E : (which == PIC_FIELD_B ? b.B : b.J);
}

}  // namespace

extern "C" {

pic_status pic_halo_floats(pic_ctx* c, int32_t box, int32_t which, int32_t side, int64_t* nfloats)
{
    CKS(halo_check(c, box, which, side));
    if (!nfloats)
        return fail(c, PIC_ERR_ARG, "nfloats is NULL");
    int p0 = 0, np = 0;
    const BoxDev& b = c->boxes_h[0];
    halo_planes(b, which, side, true, &p0, &np);
    *nfloats = 3 * (int64_t)b.px * b.py * np;
    return PIC_OK;
}

pic_status pic_halo_pack(pic_ctx* c, int32_t box, int32_t which, int32_t side, float* buf)
{
    CKS(halo_check(c, box, which, side));
    if (!buf)
        return fail(c, PIC_ERR_ARG, "buf is NULL");
    int p0 = 0, np = 0;
    const BoxDev& b = c->boxes_h[0];
    halo_planes(b, which, side, true, &p0, &np);
    CK(launch_halo_planes(b, field_of(c, which), p0, np, buf, 0, c->stream));
    return PIC_OK;
}

pic_status pic_halo_unpack(pic_ctx* c, int32_t box, int32_t which, int32_t side, const float* buf)
{
    CKS(halo_check(c, box, which, side));
    if (!buf)
        return fail(c, PIC_ERR_ARG, "buf is NULL");
    int p0 = 0, np = 0;
    const BoxDev& b = c->boxes_h[0];
    halo_planes(b, which, side, false, &p0, &np);
    CK(launch_halo_planes(b, field_of(c, which), p0, np, const_cast<float*>(buf),
                          which == PIC_FIELD_J ? 2 : 1, c->stream));
    return PIC_OK;
}

pic_status pic_migrant_bytes(pic_ctx* c, int64_t* bytes)
{
    CKS(check_ctx(c));
    if (!c->sub_z || !bytes)
        return fail(c, PIC_ERR_ARG, "migrant messages belong to a subdomain context");
    *bytes = c->mig_bytes;
    return PIC_OK;
}

pic_status pic_migrants_pack(pic_ctx* c, int32_t side, void* buf)
{
    CKS(check_ctx(c));
    if (!c->sub_z || (side != 0 && side != 1) || !buf)
        return fail(c, PIC_ERR_ARG, "bad arguments to pic_migrants_pack");
    CK(cudaMemcpyAsync(buf, c->mig + side * c->mig_bytes, (size_t)c->mig_bytes, cudaMemcpyDeviceToDevice,
                       c->stream));
    return PIC_OK;
}

pic_status pic_migrants_accept(pic_ctx* c, int32_t side, const void* buf)
{
    CKS(check_ctx(c));
    if (!c->sub_z || (side != 0 && side != 1) || !buf)
        return fail(c, PIC_ERR_ARG, "bad arguments to pic_migrants_accept");
    if (c->next_stage != PIC_STAGE_FRAMES)
        return fail(c, PIC_ERR_ARG, "migrants are accepted between the PUSH and FRAMES stages");
    CK(launch_mig_accept(make_step(c, c->parity), 0, side, static_cast<const char*>(buf), c->stream));
    return PIC_OK;
}

const char* pic_last_error(const pic_ctx* c)
{
    if (!c)
        return "null context";
    return c->err.c_str();
}

void pic_destroy(pic_ctx* c)
{
    if (!c)
        return;
    if (c->stream)
        cudaStreamSynchronize(c->stream);
    destroy_graphs(c);
    for (cudaEvent_t e : c->events)
        cudaEventDestroy(e);
    for (cudaEvent_t e : c->placeholder)
        if (e)
            cudaEventDestroy(e);
    std::vector<void*> all = c->allocs;
    for (void* p : all)
        raw_free(c, p);
    if (c->own_stream && c->stream)
        cudaStreamDestroy(c->stream);
    cudaGetLastError();
    delete c;
}

}  // extern "C"
