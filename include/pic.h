/*
 * pic.h -- C ABI of the GB300-native explicit relativistic particle-in-cell
 * step (libpic).
 *
 * The library advances one or many independent periodic 3D boxes through the
 * PIC cycle that Zenker et al. run on PIConGPU ("Performance-Portable
 * Many-Core Plasma Simulations", Sec. 2.1 and Sec. 4): field gather to the
 * particles, Boris push, charge-conserving Esirkepov current deposition, Yee
 * FDTD field update, with the particles kept in supercell-sorted frames
 * (Sec. 2.1: cells are grouped into supercells; particles live in frames of
 * as many slots as a supercell has cells, one list of frames per supercell).
 *
 * Units are normalised: c = 1, eps0 = mu0 = 1; dB/dt = -curl E and
 * dE/dt = curl B - J; momenta are u = gamma v; positions are global
 * coordinates in cell units, x in [0, N) per axis.  A macro-particle of
 * weight w and charge q carries the charge density q w S / (dx dy dz).
 * The Yee staggering is Ex(i+1/2, j, k), Ey(i, j+1/2, k), Ez(i, j, k+1/2),
 * Bx(i, j+1/2, k+1/2), By(i+1/2, j, k+1/2), Bz(i+1/2, j+1/2, k); J sits with
 * E, the charge density at the nodes.  Step order (leapfrog, B split in two
 * halves so B is known at integer time): gather E^n, B^n; Boris
 * u^{n-1/2} -> u^{n+1/2}; move; Esirkepov J^{n+1/2}; B^{n+1/2} = B^n -
 * dt/2 curl E^n; E^{n+1} = E^n + dt (curl B^{n+1/2} - J^{n+1/2});
 * B^{n+1} = B^{n+1/2} - dt/2 curl E^{n+1}.
 *
 * Threading: a context is used from one host thread at a time.  All device
 * work of a context runs on the stream given in pic_options (or on a stream
 * of its own when that is NULL).
 *
 * Errors: every call returns a pic_status and never aborts, throws or exits.
 * After any error other than PIC_ERR_ARG the context is poisoned: every later
 * call except pic_last_error and pic_destroy returns PIC_ERR_STATE.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_ctx pic_ctx; /* opaque; owned by the library */

typedef enum {
    PIC_OK = 0,
    PIC_ERR_ARG = 1,        /* bad argument: null pointer, bad size or index; ctx unchanged */
    PIC_ERR_CFL = 2,        /* dt too large: c dt must be below dx_d / 2 on every axis */
    PIC_ERR_OOM = 3,        /* the device allocator returned NULL */
    PIC_ERR_CUDA = 4,       /* a CUDA runtime call failed (message in pic_last_error) */
    PIC_ERR_FRAME_POOL = 5, /* the frame pool ran out of free frames during a step */
    PIC_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up (the push kernel waits ~2 s at most
                               for each of its tensor and bulk copies into shared memory) */
    PIC_ERR_STATE = 7,      /* the context is poisoned by an earlier error */
    PIC_ERR_CAPACITY = 8,   /* the per-step buffer of particles changing supercell overflowed */
    PIC_ERR_PARTICLE = 9    /* a particle produced a non-finite momentum or position */
} pic_status;

/* One periodic box of nx x ny x nz cells (each a multiple of the supercell
 * edge on that axis when the mixed form is used). */
typedef struct {
    int32_t nx, ny, nz;
} pic_grid;

/* One species: charge and mass in units of e and m_e (electron: -1, 1);
 * shape 1 = cloud-in-cell (linear), 2 = triangular-shaped cloud (quadratic
 * spline, the TSC of Sec. 4), 3 = piecewise cubic spline (PCS, beyond the
 * paper; mixed form only, supercells 4x4x4 with 128 threads or 8x4x4 with
 * 256, box edges >= 8; a context with a PCS species pads its fields
 * with 2 guard cells below); mobile = 0 freezes the species (it still
 * counts in the charge density and the diagnostics, and deposits no current).
 * gather: PIC_GATHER_MOMENTUM (0) interpolates every field component with
 * the particle's shape on all three axes (the paper's product of 1D
 * weights); PIC_GATHER_ENERGY (1) uses the shape one order lower along each
 * axis on which the component is staggered by half a cell (TSC -> CIC,
 * CIC -> nearest grid point), which makes the gather the transpose of the
 * Esirkepov current: for motion along one axis the field's work on the
 * particle equals the current's work on the field.  Not in the paper. */
enum { PIC_GATHER_MOMENTUM = 0, PIC_GATHER_ENERGY = 1 };
typedef struct {
    double charge, mass;
    int32_t shape;
    int32_t mobile;
    int32_t gather;
    int32_t reserved;
} pic_species;

/* Precision forms. */
enum {
    PIC_PRECISION_FP64_PLAIN = 0, /* FP64 absolute positions and fields, global atomics, no sort */
    PIC_PRECISION_MIXED = 1       /* int32 cell + FP32 offset particles in supercell frames, FP32 fields */
};

/* Field selectors for pic_write_fields / pic_read_fields. */
enum { PIC_FIELD_E = 0, PIC_FIELD_B = 1, PIC_FIELD_J = 2, PIC_FIELD_RHO = 3 };

/*
 * The field update of the mixed form (pic_options.field_update; Sec. 4: the
 * Yee solver's half step of B, step of E, half step of B):
 *   PIC_FIELD_UPDATE_IN_PLACE  three kernels per step (B half, E, B half),
 *                              each in place: 120 bytes of HBM traffic per cell;
 *   PIC_FIELD_UPDATE_FUSED     within pic_step calls of two or more steps,
 *                              one kernel per step that reads E, B, J from
 *                              one buffer pair and writes E, B into a second
 *                              one (24 bytes per padded cell, allocated at
 *                              the first step): 60 bytes per cell.  A pair of
 *                              steps goes first pair -> second -> first, so
 *                              between calls the state is in the first pair;
 *                              an odd last step, and every pic_step_stage,
 *                              uses the in-place kernels;
 *   PIC_FIELD_UPDATE_AUTO      (0) at the first step the library times one
 *                              update of each form on the context's own
 *                              fields (the fused one writes only the second
 *                              pair, the in-place one runs on a copy there)
 *                              and keeps the faster; the second pair is
 *                              freed if the in-place form wins.
 * Both forms give the same fields up to FP32 rounding of the same
 * operations.  pic_info(PIC_INFO_FIELD_UPDATE) reports the form in use.
 */
enum { PIC_FIELD_UPDATE_AUTO = 0, PIC_FIELD_UPDATE_IN_PLACE = 1, PIC_FIELD_UPDATE_FUSED = 2 };

/*
 * Supercell shape and threads per supercell (mixed form; Sec. 2.1: a
 * supercell is the unit a block of threads works on, and its shape is a
 * tuning parameter of the code).  Left 0, they are tuned by the library:
 * before the first step it times every configuration the push kernel is
 * built for that fits the boxes (sc 0,0,0: supercell shapes and thread
 * counts; threads_per_sc 0 with a given sc: thread counts) on the loaded
 * state itself -- push and frame maintenance over two sort periods after one
 * warm-up step each, in side contexts on the context's stream and allocator -- and
 * moves the context into the fastest.  The result is kept for the process
 * and reused for states of the same kind (box sizes, species, particles per
 * cell).  Until then particles sit in 4 x 4 x 4 supercells.  pic_info
 * reports the configuration in use.  A subdomain context
 * (pic_set_subdomain) keeps the configuration it was created with.
 */
typedef struct {
    int32_t precision;      /* PIC_PRECISION_* */
    int32_t sc[3];          /* supercell edge in cells (mixed form); 0,0,0 = tuned (see above) */
    int32_t threads_per_sc; /* CUDA threads per supercell work item (mixed form); 0 = tuned */
    int32_t track_ids;      /* nonzero: carry a particle id (load order) through the frames */
    int32_t use_graph;      /* nonzero: pic_step replays a captured CUDA graph of one step */
    int32_t sort_every;     /* mixed form: every this many steps the push counting-sorts each frame
                               list by nearest node (TSC) / cell (CIC, PCS) and writes it back in that
                               order; the steps between push the lists in stored order; 0 = 4,
                               1 = sort on every step (results agree up to FP32 summation order) */
    int32_t field_update;   /* mixed form, the field half of the step (Sec. 4, Yee solver), one of
                               PIC_FIELD_UPDATE_* (above); 0 = chosen at the first step */
    int32_t reserved;       /* 0 */
    int64_t pool_frames;    /* frame-pool capacity (mixed); 0 = sized at the first step from the load */
    int64_t move_capacity;  /* capacity of the per-step buffer of particles changing supercell; 0 = auto */
    /* Device allocator.  Both NULL: cudaMalloc / cudaFree.  Otherwise every
     * device buffer of the context comes from dev_alloc(bytes, alloc_ud) (it
     * must return memory usable on `stream`, 256-byte aligned, or NULL) and
     * goes back through dev_free(ptr, alloc_ud) in pic_destroy. */
    void* (*dev_alloc)(size_t bytes, void* alloc_ud);
    void (*dev_free)(void* ptr, void* alloc_ud);
    void* alloc_ud;
    void* stream;           /* cudaStream_t for all device work; NULL = a non-blocking stream the
                               context creates (graph capture needs a non-default stream) */
} pic_options;

/*
 * pic_create -- set up nboxes independent periodic boxes that share the cell
 * size dx[3], the time step dt and the species table (Sec. 2.1: the
 * simulation domain is a grid of cells grouped into supercells).
 *   grids[nboxes]   box sizes (host array, copied).
 *   dx[3]           cell edge per axis (host array, copied), > 0.
 *   dt              time step; rejected with PIC_ERR_CFL unless dt < dx_d / 2
 *                   on every axis (so no particle crosses more than half a
 *                   cell per step) and dt is below the 3D Yee Courant limit.
 *   sp[nspecies]    species table (host array, copied); 1 <= nspecies <= 8.
 *   opt             options (host, copied); NULL = all defaults.
 *   out             receives the new context.
 * Fields start at zero, boxes start empty.  On any error *out is NULL and
 * everything allocated is released.
 */
pic_status pic_create(const pic_grid* grids, int32_t nboxes, const double dx[3], double dt,
                      const pic_species* sp, int32_t nspecies, const pic_options* opt,
                      pic_ctx** out);

/*
 * pic_set_background -- a fixed, uniform charge density rho_bg for box `box`
 * (a neutralising background).  It adds to the charge density of the
 * diagnostics and carries no current.  Not in the paper (its runs load
 * electrons and ions, Sec. 4); a single-species plasma needs it to start
 * from zero fields consistently with Gauss's law.
 */
pic_status pic_set_background(pic_ctx* ctx, int32_t box, double rho_bg);

/*
 * Open boundaries along y (mixed form only; the plain form returns
 * PIC_ERR_ARG).  The paper's own runs are periodic; these are the boundary
 * steps of laser-plasma runs, on either side of the hot path.  The grid stays
 * periodic in its indexing (guards hold periodic images); the options act on
 * top of it.
 *
 * pic_set_boundary -- per box:
 *   open_y          nonzero: a particle that leaves through a y face is removed
 *                   at the end of its push (its current of that step is
 *                   deposited, folded periodically like every deposit);
 *   absorber_cells  A >= 0: damping layers of A cells at both y faces.  After
 *                   every field update each E and B component is multiplied
 *                   by exp(-sigma d^2), d in [0, 1] being the depth of its
 *                   staggered y position in the layer (0 at the layer's inner
 *                   edge, 1 at the face);
 *   absorber_sigma  sigma >= 0.
 * 2 A <= ny.  Takes effect from the next step.
 */
typedef struct {
    int32_t open_y;
    int32_t absorber_cells;
    double absorber_sigma;
} pic_boundary;
pic_status pic_set_boundary(pic_ctx* ctx, int32_t box, const pic_boundary* b);

/*
 * pic_set_antenna -- a laser antenna in box `box`: a sheet of current along x
 * on the node plane y = plane_y (the Ex positions (i+1/2, plane_y, k)), added
 * to J before the E update of every step at the current's time
 * t = (n + 1/2) dt (n = steps taken before this one):
 *   Jx += J0 exp(-((x - xc)^2 + (z - zc)^2) / w0^2) exp(-((t - t0)/tau)^2)
 *            cos(omega (t - t0)),
 *   J0 = -2 E0 cos(kappa/2) / dy,  sin(kappa/2) = (dy/dt) sin(omega dt/2),
 * so that on the Yee grid the wave leaving the sheet (to both sides) has
 * amplitude E0.  x, z, xc, zc, w0 in cell units times dx, dz; w0 <= 0: a plane
 * sheet; tau <= 0: no temporal envelope.  plane_y < 0 removes the antenna.
 * PIC_ERR_ARG when omega has no propagating wave on the grid
 * ((dy/dt) |sin(omega dt/2)| >= 1) or plane_y >= ny.
 */
typedef struct {
    int32_t plane_y;
    int32_t reserved;
    double E0, omega, w0, xc, zc, tau, t0;
} pic_antenna;
pic_status pic_set_antenna(pic_ctx* ctx, int32_t box, const pic_antenna* a);

/*
 * pic_shift_window -- moving window: box `box` moves `cells` cells towards +y.
 * Field values move down by `cells` planes, the planes entering at the top are
 * zero, particle y coordinates drop by `cells` and the particles of the bottom
 * `cells` planes are removed.  `cells` must be a positive multiple of the
 * supercell edge along y, below ny.  Fresh plasma for the top is the caller's
 * to load (pic_load_particles).
 */
pic_status pic_shift_window(pic_ctx* ctx, int32_t box, int32_t cells);

/*
 * pic_load_particles -- append n particles of species `species` to box `box`
 * (Sec. 2.1: macro particles live in a continuous domain over the cells and
 * are kept in frames of as many particles as their supercell has cells; this
 * call places each into a frame of the supercell holding its position).
 *   x[n*3]  global positions in cell units (host, FP64); wrapped
 *           periodically into [0, N) on load.
 *   u[n*3]  momenta u = gamma v, taken as u^{n-1/2} of the next step.
 *   w[n]    weights, or NULL for all ones.
 * All host arrays are read, not kept.  With track_ids the particles get ids
 * equal to their running load index within (box, species).  Returns
 * PIC_ERR_ARG for non-finite input.  Mixed form: when every array lies in one
 * page-locked host allocation (cudaHostAlloc, cudaHostRegister), the
 * conversion kernel reads it in place over the host link; otherwise the
 * arrays are staged through device memory.  The results are the same.
 */
pic_status pic_load_particles(pic_ctx* ctx, int32_t box, int32_t species, int64_t n,
                              const double* x, const double* u, const double* w);

/*
 * pic_write_fields -- overwrite field `which` (PIC_FIELD_E or PIC_FIELD_B) of
 * box `box` from f[3*nz*ny*nx] (host, FP64, component-major, x fastest), at
 * the Yee positions of the file header (Sec. 2.1: the fields live on the grid
 * of cells; Sec. 4: the Yee field solver).
 */
pic_status pic_write_fields(pic_ctx* ctx, int32_t box, int32_t which, const double* f);

/*
 * pic_step -- advance every box by nsteps full PIC cycles (step order above;
 * Sec. 4 names the cycle's algorithms: Boris pusher, Esirkepov current
 * solver, Yee field solver, TSC interpolation).
 * Blocks until the device finished, then checks the device status word:
 * PIC_ERR_FRAME_POOL, PIC_ERR_CAPACITY, PIC_ERR_PARTICLE or PIC_ERR_TIMEOUT
 * report a condition raised by a kernel.
 */
pic_status pic_step(pic_ctx* ctx, int32_t nsteps);

/*
 * pic_step_async -- as pic_step but returns once the work is enqueued on the
 * context's stream; device conditions surface at the next pic_sync.
 */
pic_status pic_step_async(pic_ctx* ctx, int32_t nsteps);

/* pic_sync -- wait for the context's stream and check the device status word (the cycle of
 * pic_step, Sec. 4). */
pic_status pic_sync(pic_ctx* ctx);

/*
 * pic_read_fields (Sec. 2.1 fields on the grid of cells; J is the Esirkepov
 * current of Sec. 4) -- copy field `which` of box `box` into out[3*nz*ny*nx]
 * (PIC_FIELD_E, _B, _J) or out[nz*ny*nx] (PIC_FIELD_RHO, the charge density
 * at the nodes including the background), host, FP64, x fastest.  J is the
 * current of the last step (J^{n+1/2}).  Mixed form, E/B/J: a page-locked
 * destination is written in place by the conversion kernel.
 */
pic_status pic_read_fields(pic_ctx* ctx, int32_t box, int32_t which, double* out);

/*
 * pic_count_particles -- number of particles of (box, species) into *n_out
 * (the sum of the counts of the species' frame lists, Sec. 2.1).
 */
pic_status pic_count_particles(pic_ctx* ctx, int32_t box, int32_t species, int64_t* n_out);

/*
 * pic_read_particles (Sec. 2.1: the frames of every supercell, in global
 * coordinates) -- copy the particles of (box, species) to host FP64
 * arrays: x[cap*3] global positions in cell units, u[cap*3], w[cap]; id[cap]
 * (optional, NULL to skip; requires track_ids).  Any of x, u, w may be NULL
 * to skip it.  The order is unspecified (frames reorder particles).  *n_out
 * receives the count; PIC_ERR_ARG if it exceeds cap (nothing is copied).
 * Mixed form: when every requested array lies in one page-locked host
 * allocation, the conversion kernel writes it in place; otherwise through
 * a device staging buffer.
 */
pic_status pic_read_particles(pic_ctx* ctx, int32_t box, int32_t species, int64_t cap,
                              double* x, double* u, double* w, int64_t* id, int64_t* n_out);

/*
 * pic_diagnostics -- FP64 reductions of box `box` into out[4] (the paper
 * prints none; these check what the step of Sec. 4 conserves: energy, charge,
 * and Gauss's law, which the charge-conserving Esirkepov current keeps):
 *   out[0] field energy   sum over cells of (E^2 + B^2)/2 * dx dy dz,
 *   out[1] kinetic energy sum over particles of w m (gamma - 1),
 *   out[2] total charge   sum of q w plus rho_bg * volume,
 *   out[3] max over nodes of |div E - rho| (Gauss's law residual).
 * Computed on the device in FP64 from the current state.
 */
pic_status pic_diagnostics(pic_ctx* ctx, int32_t box, double out[4]);

/*
 * pic_stage_times (a measurement service: the paper compares runtimes of the
 * step, Sec. 4) -- device time in milliseconds of each stage of the last
 * nsteps pic_step calls since pic_stage_timing(ctx, 1) (CUDA events on the
 * context's stream): ms[0] push+deposit, ms[1] frame maintenance,
 * ms[2] Yee update (with the J fold), ms[3] whole step; *nsteps_out
 * receives the number of steps summed.  Timing adds events between stages;
 * it is off by default.
 */
pic_status pic_stage_timing(pic_ctx* ctx, int32_t enable);
pic_status pic_stage_times(pic_ctx* ctx, double ms[4], int64_t* nsteps_out);

/*
 * pic_info (a service of this library; no counterpart in the paper) -- one
 * integer property of the context into *out:
 *   PIC_INFO_GRAPH_ACTIVE    1 if pic_step replays captured CUDA graphs (mixed form,
 *                            after the first step), else 0;
 *   PIC_INFO_KERNELS_PER_STEP number of libpic kernel launches one step makes (for a
 *                            subdomain slab: its stages and its halo / migrant calls);
 *   PIC_INFO_POOL_FRAMES     frame-pool capacity (mixed form);
 *   PIC_INFO_FRAMES_USED     frames holding particles, read from the device;
 *   PIC_INFO_MOVE_CAPACITY   capacity of the per-step buffer of particles changing supercell;
 *   PIC_INFO_STEPS           steps taken since pic_create (the time of E is STEPS * dt);
 *   PIC_INFO_HOST_DIRECT     pic_load_particles / pic_read_particles / pic_read_fields calls
 *                            of the mixed form that converted page-locked host arrays in place;
 *   PIC_INFO_SUPERCELL_X/_Y/_Z, PIC_INFO_THREADS  the supercell edges and threads per
 *                            supercell the mixed form runs with (chosen by the library's
 *                            tuner once the first step began, when pic_options left them 0);
 *   PIC_INFO_TUNE_TRIALS     configurations the tuner timed for this context (0: given in
 *                            the options, or taken from an earlier tuning in this process);
 *   PIC_INFO_FUSED_STEPS     steps since pic_create whose field update was the fused
 *                            two-buffer kernel;
 *   PIC_INFO_FIELD_UPDATE    the field update in use: PIC_FIELD_UPDATE_IN_PLACE or
 *                            PIC_FIELD_UPDATE_FUSED (PIC_FIELD_UPDATE_AUTO before the first step
 *                            of an auto context).
 * PIC_INFO_KERNELS_PER_STEP counts a step of a pic_step of two or more steps (with the
 * fused field update when it is in use: two launches fewer than the in-place kernels).
 */
enum {
    PIC_INFO_GRAPH_ACTIVE = 0,
    PIC_INFO_KERNELS_PER_STEP = 1,
    PIC_INFO_POOL_FRAMES = 2,
    PIC_INFO_FRAMES_USED = 3,
    PIC_INFO_MOVE_CAPACITY = 4,
    PIC_INFO_STEPS = 5,
    PIC_INFO_HOST_DIRECT = 6,
    PIC_INFO_SUPERCELL_X = 7,
    PIC_INFO_SUPERCELL_Y = 8,
    PIC_INFO_SUPERCELL_Z = 9,
    PIC_INFO_THREADS = 10,
    PIC_INFO_TUNE_TRIALS = 11,
    PIC_INFO_FUSED_STEPS = 12,
    PIC_INFO_FIELD_UPDATE = 13
};
pic_status pic_info(pic_ctx* ctx, int32_t key, int64_t* out);

/*
 * Domain decomposition of one periodic box into slabs along z (Sec. 2.1:
 * the simulation domain is split into local domains, one per device, each
 * a block of supercells; Sec. 1: PIConGPU runs on many GPUs).  Each process
 * holds one slab as a one-box context; the z faces of the slab exchange
 * with the neighbouring slabs (below: side 0, above: side 1) instead of
 * wrapping periodically; x and y stay periodic.  The caller moves the
 * messages between neighbours (NCCL, MPI, device copies) and runs the step
 * stage by stage:
 *   PUSH; exchange J (pic_halo_*) and migrants (pic_migrants_*); FRAMES;
 *   B_FIRST; exchange B; E; exchange E; B_SECOND; exchange B.
 * After pic_write_fields, exchange E and B once before the first step.
 *
 * pic_set_subdomain -- make box 0 of a one-box mixed-form context a z slab:
 *   enable              nonzero: z faces exchange (zero: periodic again);
 *   migrant_capacity    particles per face per step the migrant messages
 *                       hold; 0 = two per face cell.  More leavers in one
 *                       step raise PIC_ERR_CAPACITY;
 *   id_base             with track_ids: the particles loaded after this call
 *                       get ids from id_base on (per species), so that the
 *                       slabs of one box can give every particle its own id
 *                       (migrants keep theirs).
 * The slab keeps its own local coordinates: z in [0, nz) (the caller loads
 * the particles of its slab in those coordinates).  Not with open-y options
 * (PIC_ERR_ARG).  A subdomain context steps only through pic_step_stage;
 * pic_step and pic_step_async return PIC_ERR_ARG.  pic_diagnostics out[3]
 * (the Gauss residual) is taken over nodes at least 3 planes from the z
 * faces; pic_read_fields(PIC_FIELD_RHO) is exact at those nodes only.
 */
typedef struct {
    int32_t enable;
    int32_t reserved;
    int64_t migrant_capacity;
    int64_t id_base;
} pic_subdomain;
pic_status pic_set_subdomain(pic_ctx* ctx, int32_t box, const pic_subdomain* sub);

/*
 * pic_step_stage -- enqueue one stage of a PIC step on the context's stream
 * (mixed form), in the order PIC_STAGE_PUSH, _FRAMES, _B_FIRST, _E,
 * _B_SECOND (step order in the file header):
 *   PUSH      gather, Boris, move, Esirkepov deposit into a zeroed J,
 *             in-kernel frame compaction; particles leaving through a
 *             subdomain z face go to that face's migrant message;
 *   FRAMES    frame table of the next step, placing of the particles that
 *             changed supercell (accepted migrants included);
 *   B_FIRST   B^{n+1/2} = B^n - dt/2 curl E^n;
 *   E         antenna current (if any), E^{n+1} = E^n + dt (curl B - J);
 *   B_SECOND  B^{n+1} = B^{n+1/2} - dt/2 curl E^{n+1}, y absorber (if any).
 * A stage out of order returns PIC_ERR_ARG.  Device conditions surface at
 * pic_sync.  pic_step_async on a periodic context is the same five stages
 * with nothing between them.
 */
enum {
    PIC_STAGE_PUSH = 0,
    PIC_STAGE_FRAMES = 1,
    PIC_STAGE_B_FIRST = 2,
    PIC_STAGE_E = 3,
    PIC_STAGE_B_SECOND = 4
};
pic_status pic_step_stage(pic_ctx* ctx, int32_t stage);

/*
 * Field halos of a subdomain box (FP32, device memory the caller owns):
 *   which = PIC_FIELD_E or _B: the message to the neighbour on `side` holds
 *           the interior planes that neighbour keeps as guard planes; the
 *           message from the neighbour on `side` overwrites this slab's
 *           guard planes on that face;
 *   which = PIC_FIELD_J: the message to the neighbour on `side` holds this
 *           slab's guard planes on that face (current deposited by its
 *           particles into the neighbour's cells); the message from the
 *           neighbour on `side` is added into this slab's interior planes
 *           on that face.
 * Messages are whole padded planes (x and y guard columns included),
 * component-major.  pic_halo_floats gives the floats of the message sent
 * to `side`; the message received from side s has the size of the one the
 * neighbour sends to side 1 - s.  pic_halo_pack / _unpack enqueue on the
 * context's stream and return at once; `buf` must stay valid until the
 * stream reaches the copy.
 */
pic_status pic_halo_floats(pic_ctx* ctx, int32_t box, int32_t which, int32_t side, int64_t* nfloats);
pic_status pic_halo_pack(pic_ctx* ctx, int32_t box, int32_t which, int32_t side, float* buf);
pic_status pic_halo_unpack(pic_ctx* ctx, int32_t box, int32_t which, int32_t side, const float* buf);

/*
 * Migrant messages of a subdomain box: the particles that left through the
 * face `side` in the last PUSH stage, for the neighbour on that side.  A
 * message is pic_migrant_bytes bytes (device memory the caller owns): a
 * 16-byte header (int32 count, int32 capacity) and fixed-size records (species,
 * supercell x and y, cell inside the supercell, FP32 offsets, momentum and
 * weight, particle id).  pic_migrants_pack copies the message of `side`;
 * pic_migrants_accept takes the message from the neighbour on `side` (they
 * enter this slab's supercell row on that face) into the step's arrivals:
 * call it after PUSH and before FRAMES.  Both enqueue on the context's
 * stream and return at once.
 */
pic_status pic_migrant_bytes(pic_ctx* ctx, int64_t* bytes);
pic_status pic_migrants_pack(pic_ctx* ctx, int32_t side, void* buf);
pic_status pic_migrants_accept(pic_ctx* ctx, int32_t side, const void* buf);

/*
 * pic_field_energy_noalloc -- the field energy of pic_diagnostics out[0],
 * sum over cells of (E^2 + B^2) / 2 * cell_volume, computed in FP64 from
 * device arrays the caller owns, without allocating any device memory.
 * The paper has no counterpart: this is a service for callers that cannot
 * call cudaMalloc at the moment they need the number -- hosts that hand a
 * library only memory they reserved in advance, and code running where the
 * host's own rules forbid a device allocation at that point.
 *   E, B         device arrays of 3 * ncells doubles each (component-major,
 *                the layout pic_read_fields returns); read only.
 *   ncells       number of cells, 0 <= ncells <= 44,739,242; larger sizes are
 *                rejected with PIC_ERR_ARG (the fixed scratch holds 16,384
 *                partial sums of 8,192 values each).
 *   cell_volume  dx * dy * dz, > 0.
 *   out          device pointer to one double, overwritten with the result.
 *   stream       cudaStream_t to run on (NULL = legacy default stream); the
 *                call returns once the work is enqueued.
 * The partial sums live in a 128 KB array that every device loading the
 * library holds until the process exits.  The first call on a device looks
 * up that array's device address (cudaGetSymbolAddress), so make the first
 * call on each device before any stream capture.  The address is kept for
 * the life of the process: a device reset (cudaDeviceReset) between calls is
 * not supported.  Every call overwrites the partials it reads, but calls that
 * overlap on the GPU (other streams or host threads) share the array and
 * race: order them on one stream.
 * Returns PIC_ERR_ARG for bad arguments, PIC_ERR_CUDA if one of its own
 * launches fails (an error left pending by earlier calls is not consumed).
 */
pic_status pic_field_energy_noalloc(const double* E, const double* B, int64_t ncells,
                                    double cell_volume, double* out, void* stream);

/* pic_last_error -- human-readable message of the last error (never NULL); an ABI service. */
const char* pic_last_error(const pic_ctx* ctx);

/* pic_destroy -- release every resource of the context; NULL is a no-op; an ABI service. */
void pic_destroy(pic_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
