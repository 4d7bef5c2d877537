// pic_internal.cuh -- device-side data layout shared by the libpic kernels.
//
// Mixed form (int32 cell + FP32 offset particles, FP32 fields):
//
//   Fields of a box live in guard-padded arrays, one array per component,
//   x fastest: padded index = ((z+gz)*py + (y+gy))*px + (x+gx) for the real
//   cell (x, y, z).  CIC/TSC contexts: g = 1, px = nx + 4 (guards: 1 below, 3
//   above), py = ny + 3, pz = nz + 3 (1 below, 2 above).  Contexts with a PCS
//   species: g = 2, px = nx + 8 (2 below, 6 above), py = ny + 5, pz = nz + 5
//   (2 below, 3 above).  E and B guards hold periodic copies of
//   the interior (rewritten by every Yee half update); J guards collect
//   deposits that the Yee E update folds back into the periodic images.  The
//   padding lets every supercell read its E/B tile and write its J tile as one
//   regular box, 16-byte aligned along x (supercell edges are multiples of 4).
//   A box that is one z slab of a decomposed box (sub_z) keeps x and y
//   periodic; its z guards are exchanged with the neighbouring slabs instead
//   (E, B: copies of the neighbour's interior; J: sent to the neighbour and
//   added there), and particles leaving through a z face are sent on.
//
//   Particles live in frames (Sec. 2.1): a frame has S slots, S = cells per
//   supercell; attribute arrays are indexed frame * S + slot.  Each (species,
//   supercell) pair owns one list of frames; list L = species * nsc + sc.
//   The frames of list L are ftab[foff[L] + k], k < nframes[L]; its particles
//   occupy list slots 0 .. count[L]-1 densely (slot p is frame p / S, slot
//   p % S), so every frame but the last is full.  The paper keeps the frames
//   of a supercell in a doubly linked list; here the list is an index table
//   rebuilt every step by a prefix sum, so the push reads it without pointer
//   chasing.
//
//   A particle stores: cell = local cell index inside its supercell
//   (lx + LX*(ly + LY*lz)), offsets o in [0, 1) per axis, momentum u (FP32),
//   weight w.  Its global position is (supercell origin + local cell + o).
#pragma once

#include <cstdint>
#include <cuda.h>  // CUtensorMap (type only; maps are encoded through the runtime's driver entry point)
#include <cuda_runtime.h>

namespace pic {

constexpr int kMaxSpecies = 8;
constexpr int kDefaultSortEvery = 4;  // steps between sort passes of the push (mixed form)
constexpr int kYeeCellsZ = 4;         // cells per thread along z in the Yee kernels

// Device status word bits (OR-ed by kernels, read by the host after a step).
enum : unsigned {
    ST_FRAME_POOL = 1u,  // frame pool exhausted
    ST_CAPACITY = 2u,    // buffer of particles changing supercell overflowed
    ST_PARTICLE = 4u,    // non-finite momentum or a move of half a cell or more
    ST_TIMEOUT = 8u,     // a bounded device wait gave up
};

struct SpeciesDev {
    float eps;        // q dt / (2 m)   (Boris half kick factor)
    float jcoef[3];   // -q h_d / (V dt) (Esirkepov current factor; times w)
    float q;
    float m;
    int shape;        // 1 CIC, 2 TSC
    int mobile;
    float cbound;     // max over d of |jcoef[d]| * max weight: bounds |q w P T| / (V dt) terms
    int ec;           // energy-conserving gather (one order lower along staggered axes)
};

// Open-y options of a box (pic_set_boundary, pic_set_antenna).
struct OpenYDev {
    int open_y;               // particles leaving through a y face are removed
    int abs_cells;            // damping layer thickness at both y faces (0: none)
    float abs_sigma;          // damping factor exp(-sigma d^2) per step
    int ant_j;                // antenna node plane (-1: none)
    double ant_J0, ant_omega, ant_w0, ant_xc, ant_zc, ant_tau, ant_t0;
};

struct BoxDev {
    int nx, ny, nz;
    int px, py, pz;           // padded extents
    int gx, gy, gz;           // guard cells below the interior (above: p - n - g)
    int nscx, nscy, nscz;     // supercells per axis
    int sc_base;              // first global supercell id of the box
    int sub_z;                // one z slab of a decomposed box: z faces exchange, no z wrap
    float* E;                 // 3 * px*py*pz, component-major
    float* B;
    float* J;
    OpenYDev oy;
};

// Everything the mixed-form step kernels need, passed by value.
struct StepDev {
    // geometry
    int LX, LY, LZ, S, log2S;  // supercell edges, frame size
    int guard;                 // field guard cells below the interior (1, or 2 with PCS)
    int nboxes, nsc, nspecies, nlists;
    float dt;
    float move[3];            // dt / h_d
    const BoxDev* boxes;      // [nboxes]
    const CUtensorMap* tmaps; // [nboxes][2]: the E and B tile loads of the push (TMA)
    const int* sc_box;        // [nsc] box of each global supercell
    const int* items;         // [nsc] supercells in work order
    SpeciesDev sp[kMaxSpecies];
    // particle pool
    int* cell;
    float* ox;
    float* oy;
    float* oz;
    float* ux;
    float* uy;
    float* uz;
    float* w;
    int* pid;                 // null unless ids are tracked
    // lists
    int* count;               // [nlists]
    int* nframes;             // [nlists]
    const int* foff;          // [nlists] frame-table offsets (current)
    const int* ftab;          // frame table (current)
    int* foff_next;           // [nlists] (next step's table)
    int* ftab_next;
    int* narrive;             // [nlists] arrivals in this step
    int* abase;               // [nlists] first slot of this step's arrivals
    // frame pool free stack
    int* free_stack;          // [pool_frames]
    int* free_top;            // device scalar
    int* released;            // [pool_frames] frames released this step
    int pool_frames;
    // particles changing supercell this step (SoA, capacity mv_cap)
    int mv_cap;
    int* mv_count;            // device scalar
    int* mv_dest;
    int* mv_rank;
    int* mv_cell;
    float* mv_ox;
    float* mv_oy;
    float* mv_oz;
    float* mv_ux;
    float* mv_uy;
    float* mv_uz;
    float* mv_w;
    int* mv_pid;
    // particles leaving a subdomain box through a z face this step: one
    // message per face (MigHeader + mig_cap MigRec records), face f at
    // mig + f * mig_bytes
    char* mig;
    int64_t mig_bytes;
    int mig_cap;
    // scan scratch
    int4* blk_sums;           // [scan blocks]
    int4* blk_offs;           // [scan blocks]
    int4* totals;             // device scalar: frames, alloc, release, -
    int* work_counter;        // persistent-kernel work counter
    int* step_ctr;            // device step count (advanced by the frame plan)
    long long* step_no;       // steps taken since creation (advanced with step_ctr, never reset)
    int sort_every;           // the push sorts the frame lists every this many steps
    unsigned* status;         // device status word
    unsigned* wmax_bits;      // [kMaxSpecies] float bits of the largest |weight| loaded
};

// A particle that left a subdomain box through a z face (48 bytes): the
// neighbour puts it into supercell (sx, sy, its row on that face).
struct MigRec {
    int s, sx, sy, cell;
    float ox, oy, oz, ux;
    float uy, uz, w;
    int pid;
};
struct MigHeader {
    int count;  // particles written (may exceed cap: the rest were dropped)
    int cap;
    int pad[2];
};
static_assert(sizeof(MigRec) == 48 && sizeof(MigHeader) == 16, "migrant message layout");

// ---------------------------------------------------------------- helpers

__host__ __device__ inline int64_t padded_index(const BoxDev& b, int x, int y, int z)
{
    return ((int64_t)(z + b.gz) * b.py + (y + b.gy)) * b.px + (x + b.gx);
}

__host__ __device__ inline int64_t padded_cells(const BoxDev& b)
{
    return (int64_t)b.px * b.py * b.pz;
}

}  // namespace pic

// Launch helpers implemented in the kernel translation units.
namespace pic {
struct YeePlan {
    const BoxDev* boxes;  // device table
    const int* blk_off;   // device [nboxes + 1] block offsets
    int nboxes;
    int nblocks;
    float dt;
    float ih[3];
    const long long* step_no;  // steps taken, incremented before the field update of a step
    double dt_d;               // dt in FP64 (antenna time)
    double dx_d[3];            // cell edges in FP64 (antenna profile)
    const int* abs_off;        // device [nboxes + 1] block offsets of the y absorber (or null)
    int abs_nblocks;
    int antenna;               // nonzero: some box has an antenna (launch k_antenna)
    int guard;                 // field guard cells below the interior (1 or 2)
    int sub_z;                 // the (single) box is a subdomain slab: J is not folded in z
};
// The fused field update (k_yee_fused): output tiles of kFusedTX x kFusedTY
// cells z-marching through chunks of kFusedTZ planes; its E, B and J planes
// arrive by tensor loads of kFusedEX x (kFusedTY + 3) cells (x from the
// tile's x0 - guard, a 16-byte boundary of the padded row), all three
// components.
constexpr int kFusedTX = 32, kFusedTY = 8, kFusedTZ = 24, kFusedEX = 36;
struct FusedPlan {
    const BoxDev* src;        // device table of the buffers read (E^n, B^n, J)
    const BoxDev* dst;        // device table of the buffers written (E^{n+1}, B^{n+1})
    const CUtensorMap* maps;  // device [nboxes][3]: E, B, J plane maps over src's fields
    const int* blk_off;       // device [nboxes + 1] block offsets
    int nblocks;
    unsigned* status;         // ST_TIMEOUT when a tensor-load wait gave up
};
// blocks of the fused field update for one box
int fused_blocks(int nx, int ny, int nz);
// its dynamic shared memory, and the kernel attribute that allows it (call
// once, outside stream capture)
size_t fused_smem_bytes();
cudaError_t configure_yee_fused();
// the whole field update of one step from p.src into f.dst: antenna (into J),
// k_yee_fused, absorber (on dst); p supplies dt, 1/h, the antenna and absorber
cudaError_t launch_yee_fused(const YeePlan& p, const FusedPlan& f, cudaStream_t st);
cudaError_t configure_push(int LX, int LY, int LZ, int threads, int guard, int* per_sm);
// the E/B tile the push stages per supercell: row pitch px (floats), ty rows, tz planes
void push_tile_box(int LX, int LY, int LZ, int guard, int* px, int* ty, int* tz);
cudaError_t launch_push_deposit(const StepDev& d, int threads, int grid, cudaStream_t st);
int push_supported(int LX, int LY, int LZ, int threads, int guard);
size_t push_smem_bytes(int LX, int LY, int LZ, int threads, int guard);
int frame_scan_blocks(int nlists);
cudaError_t launch_frame_plan(const StepDev& d, cudaStream_t st);
cudaError_t launch_frame_apply(const StepDev& d, int place_blocks, cudaStream_t st);
// ids: per-particle ids (or null: id_base + i)
cudaError_t launch_insert_convert(const StepDev& d, int box, int species, int64_t n,
                                  const double* x, const double* u, const double* w,
                                  int id_base, const int64_t* ids, cudaStream_t st);
cudaError_t launch_read_particles(const StepDev& d, const BoxDev& hb, int box, int species,
                                  const int* list_off, double* x, double* u, double* w,
                                  int64_t* id, cudaStream_t st);
cudaError_t launch_yee_mixed_plan(const YeePlan& p, cudaStream_t st);
// one part of the field update: 0 = B half, 1 = antenna + E, 2 = B half + absorber
cudaError_t launch_yee_mixed_part(const YeePlan& p, int part, cudaStream_t st);
// planes [p0, p0 + np) (padded z) of the 3 components of F <-> buf
// ([comp][plane][py][px]); mode 0: F -> buf, 1: buf -> F, 2: F += buf
cudaError_t launch_halo_planes(const BoxDev& b, float* F, int p0, int np, float* buf, int mode,
                               cudaStream_t st);
cudaError_t launch_mig_accept(const StepDev& d, int box, int side, const char* msg, cudaStream_t st);
int absorber_blocks(const BoxDev& b);
cudaError_t launch_shift_fields(const BoxDev& b, float* F, const float* scratch, int cells,
                                cudaStream_t st);
cudaError_t launch_clear_rows(const StepDev& d, const BoxDev& hb, int rows, cudaStream_t st);
cudaError_t launch_rotate_lists(const StepDev& d, const BoxDev& hb, const int* old3, int* foff,
                                int rows, cudaStream_t st);
cudaError_t launch_fields_to_padded(const BoxDev& b, int which, const double* src,
                                    cudaStream_t st);
cudaError_t launch_fields_from_padded(const BoxDev& b, int which, double* dst, cudaStream_t st);
cudaError_t launch_diag_mixed(const StepDev& d, const BoxDev& hb, int box, double rho_bg,
                              double* rho_scratch, double* out, const double h[3],
                              cudaStream_t st);
}  // namespace pic
