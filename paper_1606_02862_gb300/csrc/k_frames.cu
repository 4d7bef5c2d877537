// k_frames.cu -- supercell frame maintenance for the mixed particle form
// (Sec. 2.1: particles live in frames of as many slots as a supercell has
// cells; each supercell owns a list of frames).
//
// After the push every list is dense again (the push fills its own holes)
// and holds count[L] particles; narrive[L] particles from neighbouring
// supercells wait in the move buffer, each with its rank among the arrivals
// of its destination list.  One step of maintenance:
//   scan_reduce / scan_top / scan_apply: an exclusive prefix sum over the
//     lists of (frames needed, frames to allocate, frames to release) gives
//     every list its place in the next frame table; scan_apply also copies
//     the kept frame indices, pops new frames off the free stack and queues
//     released ones;
//   place: every waiting particle goes to slot abase[L] + rank of its list;
//   free_push: released frames go back on the free stack.
// Loading particles from the host uses the same path: a conversion kernel
// fills the move buffer, then the maintenance places them.
#include "pic_internal.cuh"

#include <cmath>

namespace pic {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int4 operator+(int4 a, int4 b)
{
    return make_int4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

__device__ __forceinline__ int4 list_need(const StepDev& d, int L)
{
    int n_new = d.count[L] + d.narrive[L];
    int nf_new = (n_new + d.S - 1) >> d.log2S;
    int nf_old = d.nframes[L];
    return make_int4(nf_new, max(0, nf_new - nf_old), max(0, nf_old - nf_new), 0);
}

template <int NT>
__device__ int4 block_exclusive_scan(int4 v, int4* total)
{
    __shared__ int4 s_warp[NT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int4 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int4 y;
        y.x = __shfl_up_sync(0xffffffffu, x.x, o);
        y.y = __shfl_up_sync(0xffffffffu, x.y, o);
        y.z = __shfl_up_sync(0xffffffffu, x.z, o);
        y.w = __shfl_up_sync(0xffffffffu, x.w, o);
        if (lane >= o)
            x = x + y;
    }
    if (lane == 31)
        s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int4 t = lane < NT / 32 ? s_warp[lane] : make_int4(0, 0, 0, 0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int4 y;
            y.x = __shfl_up_sync(0xffffffffu, t.x, o);
            y.y = __shfl_up_sync(0xffffffffu, t.y, o);
            y.z = __shfl_up_sync(0xffffffffu, t.z, o);
            y.w = __shfl_up_sync(0xffffffffu, t.w, o);
            if (lane >= o)
                t = t + y;
        }
        if (lane < NT / 32)
            s_warp[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    int4 warp_off = wid > 0 ? s_warp[wid - 1] : make_int4(0, 0, 0, 0);
    int4 incl = x + warp_off;
    int4 excl = make_int4(incl.x - v.x, incl.y - v.y, incl.z - v.z, incl.w - v.w);
    if (total)
        *total = s_warp[NT / 32 - 1];
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const StepDev d)
{
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int4 acc = make_int4(0, 0, 0, 0);
    for (int i = 0; i < kScanItems; ++i) {
        int L = base + i;
        if (L < d.nlists)
            acc = acc + list_need(d, L);
    }
    int4 tot;
    block_exclusive_scan<kScanThreads>(acc, &tot);
    if (threadIdx.x == 0)
        d.blk_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(const StepDev d, int nblk)
{
    __shared__ int4 s_carry;
    if (threadIdx.x == 0)
        s_carry = make_int4(0, 0, 0, 0);
    __syncthreads();
    for (int b0 = 0; b0 < nblk; b0 += 1024) {
        int b = b0 + threadIdx.x;
        int4 v = b < nblk ? d.blk_sums[b] : make_int4(0, 0, 0, 0);
        int4 tot;
        int4 ex = block_exclusive_scan<1024>(v, &tot);
        int4 carry = s_carry;
        if (b < nblk)
            d.blk_offs[b] = ex + carry;
        __syncthreads();
        if (threadIdx.x == 0)
            s_carry = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *d.totals = s_carry;
        if (d.step_ctr) {
            ++*d.step_ctr;
            ++*d.step_no;
        }
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const StepDev d)
{
    const int4 tot = *d.totals;
    const int top = *d.free_top;
    if (tot.y > top) {
        // pool exhausted: report it; the step's arrivals are abandoned
        if (blockIdx.x == 0 && threadIdx.x == 0)
            atomicOr(d.status, ST_FRAME_POOL);
        return;
    }
    const int alloc_base = top - tot.y;
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int4 need[kScanItems];
    int4 acc = make_int4(0, 0, 0, 0);
    for (int i = 0; i < kScanItems; ++i) {
        int L = base + i;
        need[i] = L < d.nlists ? list_need(d, L) : make_int4(0, 0, 0, 0);
        acc = acc + need[i];
    }
    int4 off = block_exclusive_scan<kScanThreads>(acc, nullptr) + d.blk_offs[blockIdx.x];
    for (int i = 0; i < kScanItems; ++i) {
        int L = base + i;
        if (L >= d.nlists)
            break;
        const int nf_new = need[i].x;
        const int nf_old = d.nframes[L];
        const int* src = d.ftab + d.foff[L];
        int* dst = d.ftab_next + off.x;
        const int keep = min(nf_old, nf_new);
        for (int k = 0; k < keep; ++k)
            dst[k] = src[k];
        for (int k = nf_old; k < nf_new; ++k)
            dst[k] = d.free_stack[alloc_base + off.y + (k - nf_old)];
        for (int k = nf_new; k < nf_old; ++k)
            d.released[off.z + (k - nf_new)] = src[k];
        d.foff_next[L] = off.x;
        d.nframes[L] = nf_new;
        const int c = d.count[L];
        d.abase[L] = c;
        d.count[L] = c + d.narrive[L];
        d.narrive[L] = 0;
        off = off + need[i];
    }
}

__global__ void k_place(const StepDev d)
{
    const int4 tot = *d.totals;
    if (tot.y > *d.free_top)
        return;
    const int n = min(*d.mv_count, d.mv_cap);
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
        const int L = d.mv_dest[m];
        const int slot = d.abase[L] + d.mv_rank[m];
        const int frame = d.ftab_next[d.foff_next[L] + (slot >> d.log2S)];
        const int64_t idx = (int64_t)frame * d.S + (slot & (d.S - 1));
        d.cell[idx] = d.mv_cell[m];
        d.ox[idx] = d.mv_ox[m];
        d.oy[idx] = d.mv_oy[m];
        d.oz[idx] = d.mv_oz[m];
        d.ux[idx] = d.mv_ux[m];
        d.uy[idx] = d.mv_uy[m];
        d.uz[idx] = d.mv_uz[m];
        d.w[idx] = d.mv_w[m];
        if (d.pid)
            d.pid[idx] = d.mv_pid[m];
    }
}

__global__ void __launch_bounds__(1024) k_free_push(const StepDev d)
{
    const int4 tot = *d.totals;
    const int top = *d.free_top;
    if (tot.y > top)
        return;
    const int base = top - tot.y;
    for (int i = threadIdx.x; i < tot.z; i += blockDim.x)
        d.free_stack[base + i] = d.released[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        *d.free_top = base + tot.z;
        *d.mv_count = 0;
    }
}

// Moving window, part 1: empty the lists of the bottom `rows` supercell
// rows of a box (every species); the next maintenance pass releases their
// frames.
__global__ void k_clear_rows(const StepDev d, const BoxDev b, int rows)
{
    const int per_species = b.nscx * rows * b.nscz;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < d.nspecies * per_species;
         t += gridDim.x * blockDim.x) {
        const int s = t / per_species, r = t % per_species;
        const int scx = r % b.nscx, scy = (r / b.nscx) % rows, scz = r / (b.nscx * rows);
        d.count[s * d.nsc + b.sc_base + (scz * b.nscy + scy) * b.nscx + scx] = 0;
    }
}

// Moving window, part 2: the list of row scy takes over the list (count,
// frames, frame-table offset) of row scy + rows, cyclically; the rows that
// were emptied in part 1 come round to the top.  old3 = copies of count,
// nframes and foff (nlists each), taken before the kernel.
__global__ void k_rotate_lists(const StepDev d, const BoxDev b, const int* old3, int* foff, int rows)
{
    const int nbox = b.nscx * b.nscy * b.nscz;
    const int* count_old = old3;
    const int* nframes_old = old3 + d.nlists;
    const int* foff_old = old3 + 2 * d.nlists;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < d.nspecies * nbox;
         t += gridDim.x * blockDim.x) {
        const int s = t / nbox, loc = t % nbox;
        const int scx = loc % b.nscx, scy = (loc / b.nscx) % b.nscy, scz = loc / (b.nscx * b.nscy);
        const int sy = (scy + rows) % b.nscy;
        const int L = s * d.nsc + b.sc_base + loc;
        const int Ls = s * d.nsc + b.sc_base + (scz * b.nscy + sy) * b.nscx + scx;
        d.count[L] = count_old[Ls];
        d.nframes[L] = nframes_old[Ls];
        foff[L] = foff_old[Ls];
    }
}

cudaError_t launch_clear_rows(const StepDev& d, const BoxDev& hb, int rows, cudaStream_t st)
{
    k_clear_rows<<<256, 256, 0, st>>>(d, hb, rows);
    return cudaGetLastError();
}

cudaError_t launch_rotate_lists(const StepDev& d, const BoxDev& hb, const int* old3, int* foff,
                                int rows, cudaStream_t st)
{
    k_rotate_lists<<<256, 256, 0, st>>>(d, hb, old3, foff, rows);
    return cudaGetLastError();
}

int frame_scan_blocks(int nlists) { return (nlists + kScanTile - 1) / kScanTile; }

cudaError_t launch_frame_plan(const StepDev& d, cudaStream_t st)
{
    const int nblk = frame_scan_blocks(d.nlists);
    k_scan_reduce<<<nblk, kScanThreads, 0, st>>>(d);
    k_scan_top<<<1, 1024, 0, st>>>(d, nblk);
    return cudaGetLastError();
}

cudaError_t launch_frame_apply(const StepDev& d, int place_blocks, cudaStream_t st)
{
    const int nblk = frame_scan_blocks(d.nlists);
    k_scan_apply<<<nblk, kScanThreads, 0, st>>>(d);
    k_place<<<place_blocks, 256, 0, st>>>(d);
    k_free_push<<<1, 1024, 0, st>>>(d);
    return cudaGetLastError();
}

// ------------------------------------------------------------ subdomain migrants

// The migrant message of the neighbouring slab on face `side` of box `box`
// (a one-box subdomain context): every record joins this step's arrivals
// (the move buffer) in supercell (sx, sy, row on that face), where the frame
// plan and k_place then put it like any particle that changed supercell.
__global__ void k_mig_accept(const StepDev d, int box, int side, const char* msg)
{
    const BoxDev b = d.boxes[box];
    const MigHeader h = *reinterpret_cast<const MigHeader*>(msg);
    const int n = min(h.count, h.cap);
    const MigRec* rec = reinterpret_cast<const MigRec*>(msg + sizeof(MigHeader));
    const int sz = side == 0 ? 0 : b.nscz - 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const MigRec r = rec[i];
        if (r.s < 0 || r.s >= d.nspecies || r.sx < 0 || r.sx >= b.nscx || r.sy < 0 || r.sy >= b.nscy ||
            r.cell < 0 || r.cell >= d.S) {
            atomicOr(d.status, ST_PARTICLE);  // a malformed record is dropped
            continue;
        }
        const int L = r.s * d.nsc + b.sc_base + (sz * b.nscy + r.sy) * b.nscx + r.sx;
        const int m = atomicAdd(d.mv_count, 1);
        if (m >= d.mv_cap) {
            atomicOr(d.status, ST_CAPACITY);
            continue;
        }
        d.mv_rank[m] = atomicAdd(d.narrive + L, 1);
        d.mv_dest[m] = L;
        d.mv_cell[m] = r.cell;
        d.mv_ox[m] = r.ox;
        d.mv_oy[m] = r.oy;
        d.mv_oz[m] = r.oz;
        d.mv_ux[m] = r.ux;
        d.mv_uy[m] = r.uy;
        d.mv_uz[m] = r.uz;
        d.mv_w[m] = r.w;
        if (d.pid)
            d.mv_pid[m] = r.pid;
    }
}

cudaError_t launch_mig_accept(const StepDev& d, int box, int side, const char* msg, cudaStream_t st)
{
    k_mig_accept<<<256, 256, 0, st>>>(d, box, side, msg);
    return cudaGetLastError();
}

// ------------------------------------------------------------ load / read

// Host particles (FP64, n x 3 global cell coordinates) -> move buffer.  A
// block takes 256 particles at a time: their x, u and w runs come into
// shared memory word by word across the threads (each warp load is 256
// contiguous bytes: the source may be page-locked host memory read over the
// host link), then each thread converts one particle.
constexpr int kInsertBlock = 256;

__global__ void __launch_bounds__(kInsertBlock) k_insert_convert(const StepDev d, int box, int species, int n,
                                                                 const double* x, const double* u,
                                                                 const double* w, int id_base,
                                                                 const int64_t* ids)
{
    __shared__ double sx[3 * kInsertBlock], su[3 * kInsertBlock], sw[kInsertBlock];
    const BoxDev b = d.boxes[box];
    const int Nd[3] = {b.nx, b.ny, b.nz};
    const int Ld[3] = {d.LX, d.LY, d.LZ};
    for (int64_t base = (int64_t)blockIdx.x * kInsertBlock; base < n; base += (int64_t)gridDim.x * kInsertBlock) {
        const int m = (int)(n - base < kInsertBlock ? n - base : kInsertBlock);
        __syncthreads();  // the previous group's reads of the stage are done
        for (int j = threadIdx.x; j < 3 * m; j += kInsertBlock) {
            sx[j] = x[3 * base + j];
            su[j] = u[3 * base + j];
        }
        if (threadIdx.x < m)
            sw[threadIdx.x] = w ? w[base + threadIdx.x] : 1.0;
        __syncthreads();
        if (threadIdx.x >= m)
            continue;
        const int t = threadIdx.x;
        const int i = (int)(base + t);
        int scd[3], lc[3];
        float o[3];
        bool bad = false;
        for (int a = 0; a < 3; ++a) {
            double v = sx[3 * t + a];
            if (!isfinite(v) || !isfinite(su[3 * t + a]))
                bad = true;
            double N = (double)Nd[a];
            v = v - N * floor(v / N);
            if (!(v < N))
                v = 0.0;
            if (!(v >= 0.0))
                v = 0.0;
            int ci = (int)floor(v);
            ci = min(max(ci, 0), Nd[a] - 1);
            float of = (float)(v - (double)ci);
            of = fminf(fmaxf(of, 0.0f), 0.99999994f);
            o[a] = of;
            scd[a] = ci / Ld[a];
            lc[a] = ci - scd[a] * Ld[a];
        }
        const double wv = sw[t];
        if (!isfinite(wv))
            bad = true;
        if (bad)
            atomicOr(d.status, ST_PARTICLE);
        else
            atomicMax(d.wmax_bits + species, __float_as_uint(fabsf((float)wv)));
        const int sc = b.sc_base + (scd[2] * b.nscy + scd[1]) * b.nscx + scd[0];
        const int L = species * d.nsc + sc;
        d.mv_dest[i] = L;
        d.mv_rank[i] = bad ? 0 : atomicAdd(d.narrive + L, 1);
        d.mv_cell[i] = lc[0] + d.LX * (lc[1] + d.LY * lc[2]);
        d.mv_ox[i] = o[0];
        d.mv_oy[i] = o[1];
        d.mv_oz[i] = o[2];
        d.mv_ux[i] = (float)su[3 * t + 0];
        d.mv_uy[i] = (float)su[3 * t + 1];
        d.mv_uz[i] = (float)su[3 * t + 2];
        d.mv_w[i] = (float)wv;
        if (d.mv_pid)
            d.mv_pid[i] = ids ? (int)ids[i] : id_base + i;
    }
}

cudaError_t launch_insert_convert(const StepDev& d, int box, int species, int64_t n,
                                  const double* x, const double* u, const double* w, int id_base,
                                  const int64_t* ids, cudaStream_t st)
{
    int blocks = (int)std::min<int64_t>((n + kInsertBlock - 1) / kInsertBlock, 4096);
    if (blocks > 0)
        k_insert_convert<<<blocks, kInsertBlock, 0, st>>>(d, box, species, (int)n, x, u, w, id_base, ids);
    return cudaGetLastError();
}

// One CTA per supercell of the box: copy its particles to FP64 global form
// at list_off[sc] (exclusive prefix of the counts, host-computed).  Thread j
// writes word j of the supercell's run of x (and of u), so that every warp
// store covers 256 contiguous bytes: the destination may be page-locked host
// memory written over the host link, where partial sectors cost.
__global__ void k_read_particles(const StepDev d, int box, int species, const int* list_off,
                                 double* x, double* u, double* w, int64_t* id)
{
    const BoxDev b = d.boxes[box];
    const int loc = blockIdx.x;
    const int g = b.sc_base + loc;
    const int L = species * d.nsc + g;
    const int n = d.count[L];
    const int scx = loc % b.nscx, scy = (loc / b.nscx) % b.nscy, scz = loc / (b.nscx * b.nscy);
    const int* ft = d.ftab + d.foff[L];
    const int64_t o0 = list_off[loc];
    for (int j = threadIdx.x; j < 3 * n; j += blockDim.x) {
        const int p = j / 3, a = j - 3 * p;
        const int64_t idx = (int64_t)ft[p >> d.log2S] * d.S + (p & (d.S - 1));
        if (x) {
            const int cell = d.cell[idx];
            const int gc = a == 0 ? scx * d.LX + cell % d.LX
                                  : (a == 1 ? scy * d.LY + (cell / d.LX) % d.LY : scz * d.LZ + cell / (d.LX * d.LY));
            x[3 * o0 + j] = (double)gc + (double)(a == 0 ? d.ox : (a == 1 ? d.oy : d.oz))[idx];
        }
        if (u)
            u[3 * o0 + j] = (double)(a == 0 ? d.ux : (a == 1 ? d.uy : d.uz))[idx];
    }
    if (w || id)
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            const int64_t idx = (int64_t)ft[p >> d.log2S] * d.S + (p & (d.S - 1));
            if (w)
                w[o0 + p] = (double)d.w[idx];
            if (id)
                id[o0 + p] = d.pid ? (int64_t)d.pid[idx] : -1;
        }
}

cudaError_t launch_read_particles(const StepDev& d, const BoxDev& hb, int box, int species,
                                  const int* list_off, double* x, double* u, double* w,
                                  int64_t* id, cudaStream_t st)
{
    const int nsc_box = hb.nscx * hb.nscy * hb.nscz;
    if (nsc_box == 0)
        return cudaSuccess;
    k_read_particles<<<nsc_box, 128, 0, st>>>(d, box, species, list_off, x, u, w, id);
    return cudaGetLastError();
}

}  // namespace pic
