/*
 * lbm.h -- C ABI of the GB300 two-component Shan-Chen D3Q19 library.
 *
 * The library implements the time step that the hybrid pore-network / lattice
 * Boltzmann method of Montella, Yuan, Chareyre and Gens spends its time in:
 * pull streaming with half-way bounce-back (Eq. 1, left-hand side), moments
 * (Eqs. 2-3), the Shan-Chen inter-component force (Eq. 4, read with psi = rho
 * and the lattice weights), wall adhesion, the velocity-shift BGK collision
 * (Eq. 1, right-hand side) and reservoir layers whose densities are raised step
 * by step to drive drainage (Sec. 2.2.2).  The measurements return the bulk
 * phase pressures of the equation of state (Eq. 5), the capillary pressure and
 * the saturation from which the entry pressure p_c^e (the largest p_c reached
 * during invasion, Sec. 2.2.2) is read.
 *
 * Conventions shared by every call:
 *  - Lattice units.  Cell (x, y, z) has its centre at (x, y, z); cell index
 *    c = (z * ny + y) * nx + x.  N = nx * ny * nz.
 *  - Component 0 is the wetting fluid, component 1 the non-wetting fluid.
 *  - D3Q19 order of the populations: k = 0 rest; 1..6 = (+x, -x, +y, -y, +z, -z);
 *    7..10 = (+x+y, -x-y, +x-y, -x+y); 11..14 = (+x+z, -x-z, +x-z, -x+z);
 *    15..18 = (+y+z, -y-z, +y-z, -y+z).  Opposite pairs are (1,2), (3,4), ...
 *  - Mask bytes: bit 0 solid, bit 1 adhesive (grain; meaningful with bit 0),
 *    bit 2 membrane (solid for the non-wetting fluid only), bit 3 inlet
 *    reservoir layer, bit 4 outlet reservoir layer.
 *  - Cells beyond a non-periodic box edge are neutral (non-adhesive) walls.
 *  - Every pointer argument is a HOST pointer unless stated otherwise; inputs
 *    are copied during the call and stay owned by the caller.  Device memory is
 *    allocated and owned by the library and released by lbm_destroy.
 *  - Every int-returning call returns LBM_OK (0) or a negative LBM_ERR_* code
 *    and then lbm_last_error() describes the failure (thread-local string).
 *    No C++ exception crosses this boundary.
 *  - A domain is not thread-safe; distinct domains may run on distinct streams.
 */
#ifndef LBM_H_
#define LBM_H_

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_ERR_ARG (-1)       /* invalid argument (null pointer, bad size, bad enum)   */
#define LBM_ERR_OOM (-2)       /* device or host allocation failed                      */
#define LBM_ERR_CUDA (-3)      /* a CUDA runtime call failed                            */
#define LBM_ERR_TIMEOUT (-4)   /* a bounded wait for device work ran out                */
#define LBM_ERR_NONFINITE (-5) /* a measurement met NaN/Inf or negative densities       */
#define LBM_ERR_STATE (-6)     /* call not valid in the domain's current state          */

#define LBM_MASK_SOLID 1
#define LBM_MASK_ADHESIVE 2
#define LBM_MASK_MEMBRANE 4
#define LBM_MASK_INLET 8
#define LBM_MASK_OUTLET 16

typedef struct lbm_domain lbm_domain; /* opaque, library-owned */

/* Model parameters (lattice units). */
typedef struct {
    double tau[2];        /* BGK relaxation time per component (> 0.5)                 */
    double G;             /* Shan-Chen inter-component strength G_12 = G_21 (Eq. 4)     */
    double G_ads[2];      /* wall adhesion strength per component (< 0 attracts)        */
    double body_force[3]; /* acceleration g; the body force on component s is rho_s g   */
    double rho_major;     /* density of the majority fluid of a phase (e.g. 2.0)        */
    double rho_minor;     /* density of the dissolved other fluid (e.g. 0.06)           */
    int precision;        /* storage of the populations: 0 = FP32; 1 = FP16 and 2 = BF16
                             deviations (pairs of both components per direction, taken
                             against the reading cell's previous density; collision in
                             FP32).  lbm_run_throat_batch always uses FP32.            */
    int periodic[3];      /* 1 = periodic along x, y, z                                 */
    int reservoirs;       /* 1 = inlet layer z = 0 (non-wetting reservoir) and outlet
                             layer z = nz-1 (wetting reservoir)                          */
    int membrane_layers;  /* fluid layers just above the outlet layer that let only the
                             wetting fluid pass (porous plate); 0 = none                 */
    int prism_clip;       /* 1 = cells outside the triangular prism of the first three
                             spheres are neutral walls (throat domain, Sec. 2.2.2)       */
} lbm_params;

/* Observables of the state at the current time level (Eq. 5 for pressures).
 *   interior fluid = not solid, not membrane, not a reservoir layer;
 *   S_w = #(interior cells with rho_w > rho_nw) / #(interior cells);
 *   interface cells: |phi| < 0.5 with phi = (rho_w - rho_nw)/(rho_w + rho_nw);
 *   p_w, p_nw: mean Eq. 5 pressure over interior cells with phi > 0.9 / < -0.9;
 *   p_c = p_nw - p_w (NaN when a phase has no bulk cell);
 *   p_in, p_out: mean pressure over the inlet / outlet layers; p_c_res = p_in - p_out.
 * Sums are accumulated in FP64 on the device. */
typedef struct {
    double mass[2];
    double p_w, p_nw, p_c;
    double p_in, p_out, p_c_res;
    double S_w;
    long long n_fluid, n_w, n_interface, n_bulk_w, n_bulk_nw, n_in, n_out;
    long long n_nonfinite, n_negative;
    int status_flags; /* bit 0: NaN/Inf density seen; bit 1: negative density seen */
} lbm_measurement;

/* lbm_create_domain -- voxelise spheres into a box and allocate a domain
 * (Sec. 2.2.2 throat domain when prism_clip = 1; the fully resolved sample
 * otherwise).
 *   spheres   n_spheres x 4 doubles (cx, cy, cz, r), lattice units; a cell is
 *             grain (solid + adhesive) when |centre - c| <= r.  May be NULL when
 *             n_spheres = 0.
 *   box       (nx, ny, nz), each >= 1.
 *   stream    cudaStream_t the domain's work is queued on (NULL = legacy stream).
 * The populations start at the rest equilibrium of rho_major wetting fluid
 * (with rho_minor non-wetting) and, on the inlet layer, the reverse.
 * Returns LBM_ERR_ARG for bad sizes or params, LBM_ERR_OOM when device memory
 * runs out. */
int lbm_create_domain(const lbm_params* params, const double* spheres, int n_spheres,
                      const int box[3], void* stream, lbm_domain** out);

/* lbm_create_domain_mask -- as lbm_create_domain, from an explicit mask
 * (N bytes, layout above) instead of spheres; prism_clip, reservoirs and
 * membrane_layers in params are ignored (the mask already carries them). */
int lbm_create_domain_mask(const lbm_params* params, const unsigned char* mask, const int box[3],
                           void* stream, lbm_domain** out);

/* lbm_set_densities -- reset the populations to the rest equilibrium of the
 * given densities: rho (2 x N doubles, component-major).  Values at cells where
 * a component is not fluid are ignored.  Resets the step counter. */
int lbm_set_densities(lbm_domain* d, const double* rho);

/* lbm_set_pressure_bc -- densities imposed on the reservoir layers from the
 * next step on: inlet (rho_minor, rho_in_nw), outlet (rho_out_w, rho_minor)
 * (Sec. 2.2.2: the inlet/outlet densities are adjusted to raise p_c). */
int lbm_set_pressure_bc(lbm_domain* d, double rho_in_nw, double rho_out_w);

/* lbm_step -- queue n_steps fused time steps on the domain's stream
 * (asynchronous; n_steps >= 0).  Whole chunks of 64 steps replay a CUDA graph
 * captured on first use (one per starting buffer, recaptured after
 * lbm_set_tile); the remainder is launched step by step.  Results are the same
 * either way, bit for bit. */
int lbm_step(lbm_domain* d, int n_steps);

/* lbm_measure -- observables of the current state (synchronises the domain's
 * stream, bounded by a 60 s wait: LBM_ERR_TIMEOUT).  Returns LBM_ERR_NONFINITE
 * (with *out filled) when NaN/Inf or negative densities were found. */
int lbm_measure(lbm_domain* d, lbm_measurement* out);

/* lbm_get_density_at -- (rho_w, rho_nw) of one cell of the current state
 * (synchronising); LBM_ERR_ARG outside the box. */
int lbm_get_density_at(lbm_domain* d, int x, int y, int z, double rho_out[2]);

/* One pressure increment of a drainage ladder. */
typedef struct {
    double rho_in_nw;      /* inlet non-wetting density of the increment              */
    double p_c, p_c_res;   /* bulk-phase and reservoir capillary pressure (lbm_measure) */
    double S_w, p_w, p_nw;
    double phi_probe;      /* (rho_w - rho_nw)/(rho_w + rho_nw) at the probe cell       */
    long long n_interface;
} lbm_increment;

/* lbm_run_drainage -- the pressure ladder of Sec. 2.2.2: for increment i the
 * inlet reservoir is set to (rho_minor, rho_in_nw[i]) and the outlet to
 * (rho_out_w, rho_minor), n_steps time steps run (replayed CUDA graphs of 64
 * steps), and the domain is measured into rows[i].  The throat counts as
 * invaded at the first increment after which phi < 0 at the probe cell (x, y, z);
 * p_c^e is the largest p_c (bulk-phase) up to and including that increment --
 * the maximum capillary pressure reached during invasion -- the first maximiser
 * winning ties; *p_ce = +inf and *invaded_at = -1 when the probe never turned
 * non-wetting.  rows holds n_incr entries (caller-owned).  Synchronising. */
int lbm_run_drainage(lbm_domain* d, const double* rho_in_nw, int n_incr, int n_steps, double rho_out_w,
                     const int probe[3], lbm_increment* rows, double* p_ce, int* invaded_at);

/* Pressure ladder shared by every throat of a batch. */
typedef struct {
    int n_incr;               /* number of increments (>= 1)                          */
    int n_steps;              /* time steps per increment (>= 0)                      */
    const double* rho_in_nw;  /* n_incr inlet non-wetting densities (host, caller's)  */
    double rho_out_w;         /* outlet wetting density                               */
    int per_throat;           /* lbm_run_throat_batch: 1 = rho_in_nw holds one ladder
                                 per throat, n x n_incr throat-major; 0 = one ladder
                                 for all throats                                      */
    int batch_form;           /* lbm_run_throat_batch: LBM_BATCH_AUTO, _PERSISTENT or
                                 _PER_STEP (below)                                    */
    int march_threads;        /* LBM_BATCH_MARCH: threads per CTA, 128 (four CTAs an
                                 SM), 256 (two), 384 or 512 (one); 0: the default,
                                 LBM_MARCH_THREADS                                     */
    int march_planes;         /* LBM_BATCH_MARCH: planes per chunk, 1 .. 64 (0: the
                                 default, LBM_MARCH_PLANES)                            */
} lbm_schedule;

/* Forms of lbm_run_throat_batch.  PERSISTENT: one launch per increment, a CTA
 * takes a whole throat off a work counter and runs all of the increment's steps
 * on it (no grid-wide synchronisation; best when the throats outnumber the CTAs
 * that fit on the GPU).  PER_STEP: one launch per time step over a work list of
 * every throat's active tiles and z segments, so that a few large throats still
 * fill the GPU.  CELLS: the populations of the non-solid cells only, stored
 * compactly after streaming; two launches per time step over that cell list,
 * one thread per cell (a density pass, then the collision, which pushes each
 * value to the cell it streams to), so that the grain inside the throat boxes
 * (most of a box) costs neither lanes, traffic nor memory.  MARCH: the same
 * cell list in one launch per time step, a CTA per chunk of up to
 * march_planes planes of a throat, which computes the densities of a plane and steps the plane below
 * it right after (a plane's pairs are read a second time from cache, not from
 * DRAM).  All forms give bit-identical rows.  AUTO is CELLS. */
#define LBM_BATCH_AUTO 0
#define LBM_BATCH_PERSISTENT 1
#define LBM_BATCH_PER_STEP 2
#define LBM_BATCH_CELLS 3
#define LBM_BATCH_MARCH 4
/* Defaults of the marching form's launch shape (lbm_schedule.march_threads,
 * .march_planes). */
#define LBM_MARCH_THREADS 256
#define LBM_MARCH_PLANES 16

/* Per-throat outcome of a batch. */
typedef struct {
    double p_ce;         /* entry capillary pressure (rule of lbm_run_drainage); +inf if not invaded */
    int invaded_at;      /* increment of invasion, -1 if none                                      */
    int dims[3];         /* throat box (nx, ny, nz)                                                */
    int probe[3];        /* probe cell, -1s if the probe plane holds no fluid                      */
    long long n_fluid;   /* interior fluid cells                                                   */
} lbm_throat_result;

/* lbm_throat_geometry -- the throat domain of Sec. 2.2.2 for three spheres
 * (spheres3: 3 x (cx, cy, cz, r), any frame): a box in the frame of the three
 * centres (x along c1 - c0, z along the normal of their plane; cell (i, j, k)
 * at local (x0 + i, y0 + j, -ceil(rmax) + k) with x0, y0 the floors of the
 * centres' local minima), grain inside the spheres, neutral walls outside the
 * triangular prism whose walls pass through pairs of centres orthogonally to
 * their plane, inlet layer k = 0 and outlet layer k = nz - 1.  Fills dims_out;
 * when mask_out is not NULL also the nx*ny*nz mask bytes and probe_out (the
 * fluid cell of plane nz - 3 farthest from the sphere surfaces, where invasion
 * is detected).  LBM_ERR_ARG for collinear centres or boxes beyond 512. */
int lbm_throat_geometry(const double* spheres3, int dims_out[3], unsigned char* mask_out, int probe_out[3]);

/* lbm_throat_lattice_features -- what the lattice makes of each throat, for the
 * surrogate: the throat boxes of lbm_throat_geometry are voxelised (host, all
 * cores) and described by LBM_THROAT_LATTICE_FEATURES numbers each (row t of
 * out, n x 14 doubles, caller-owned).  With A(k) the non-solid cells of plane k
 * and the interior planes k = 1 .. nz - 2 (all planes when nz < 3), ordered by
 * (A, k) ascending, k* the first of them:
 *    0-2  nx, ny, nz
 *    3    non-solid fraction of the box
 *    4    A(k*)                       5  sqrt(A(k*) / pi)
 *    6    mean A over interior planes 7  k* / nz
 *    8    lattice incircle of plane k*: the largest Euclidean distance from a
 *         non-solid cell to the nearest solid cell of the same plane
 *    9-10 max and mean of that incircle over the first three planes
 *    11   A(k*) / max(P, 1)           12 P: non-solid cells of plane k* with a
 *         solid or out-of-plane 4-neighbour
 *    13   mean of the first three A
 * The entry pressure of a throat follows its narrowest section (Young-Laplace);
 * these say how the lattice resolves that section.  Errors as
 * lbm_throat_geometry (LBM_ERR_ARG for a bad throat; nothing is written). */
#define LBM_THROAT_LATTICE_FEATURES 14
int lbm_throat_lattice_features(const double* throats, int n, double* out);

/* lbm_run_throat_batch -- the per-throat simulations of the hybrid method
 * (Sec. 2.2.2: one LBM run per pore throat, p_c^e from its drainage ladder) for
 * n throats at once: each throat's box (lbm_throat_geometry) starts filled with
 * wetting fluid, then runs the schedule's ladder exactly as lbm_run_drainage
 * would on that box alone.  All throats run together in one device arena, in the
 * form sched->batch_form selects (LBM_BATCH_CELLS by default: the throats'
 * non-solid cells as one list, two launches per time step; see the forms
 * above); one increment is captured as a CUDA graph and relaunched.  Every form
 * gives the same rows bit for bit.  The host set-up (voxelising the boxes,
 * building the lists) runs on all host cores.
 *   throats   n x 3 x 4 doubles (host)
 *   params    tau, G, G_ads, body_force, rho_major, rho_minor are used
 *   results   n entries (host, caller-owned)
 *   rows      n x n_incr increments, throat-major (host, caller-owned)
 *   stream    cudaStream_t (NULL = legacy stream); the call synchronises it.
 * Device memory is allocated for the call and released before it returns. */
int lbm_run_throat_batch(const double* throats, int n, const lbm_params* params, const lbm_schedule* sched,
                         lbm_throat_result* results, lbm_increment* rows, void* stream);

/* lbm_run_throat_batch_refined -- lbm_run_throat_batch (results, rows as
 * there), then p_c^e below the ladder step: every throat invaded at increment
 * k >= 1 runs again with the same levels up to k - 1 (the same state, the run
 * being deterministic) followed by n_fine equal sub-steps from level k - 1 to
 * level k (sched->n_steps each, the ladder padded with level k to a common
 * length), and p_ce_fine[t] is that run's p_c^e (the rule of
 * lbm_run_drainage).  Throats invaded at increment 0 keep the coarse p_c^e, and
 * so does a throat the second run does not invade; +inf where the first run
 * did not invade.  n_fine = 1 returns the coarse values.  Per-throat ladders
 * (sched->per_throat) are refined each on its own levels.  p_ce_fine: n
 * doubles (host, caller-owned).  LBM_ERR_ARG for n_fine < 1. */
int lbm_run_throat_batch_refined(const double* throats, int n, const lbm_params* params, const lbm_schedule* sched,
                                 int n_fine, lbm_throat_result* results, lbm_increment* rows, double* p_ce_fine,
                                 void* stream);

/* ---------------------------------------------------------------------------
 * Pore network (Sec. 2.2.1 pore-space decomposition, Sec. 2.2.2 fluid
 * displacement, Sec. 3.1.1 drainage of the sample).  Host computations; the
 * entry pressures they consume come from lbm_run_throat_batch (or the
 * surrogate, or the incircle estimate).
 * ------------------------------------------------------------------------- */
#define LBM_PN_INLET (-1)   /* throat_pores second entry: the non-wetting reservoir */
#define LBM_PN_OUTLET (-2)  /* throat_pores second entry: the wetting reservoir (behind the membrane) */

/* lbm_regular_triangulation -- the regular triangulation of the sphere centres
 * weighted by the squared radii (Sec. 2.2.1: tetrahedra are pore bodies, their
 * facets pore throats; for equal radii it is the Delaunay tetrahedralisation),
 * by Bowyer-Watson insertion in double precision.
 *   spheres   n x (cx, cy, cz, r), n >= 4, non-overlapping spheres (then every
 *             centre is a vertex; a redundant weighted point would be skipped).
 *   tets_out  capacity x 4 sphere indices (host, caller-owned), each
 *             tetrahedron positively oriented; may be NULL when capacity = 0,
 *             which only counts.
 *   n_tets    the number of tetrahedra.
 * LBM_ERR_ARG for bad input, a degenerate (flat) configuration, or a capacity
 * below the count (*n_tets still holds it). */
int lbm_regular_triangulation(const double* spheres, int n, int* tets_out, int capacity, int* n_tets);

/* lbm_packing_throats -- the pore throats of a packing (Sec. 2.2.1): the facets
 * that two tetrahedra of lbm_regular_triangulation share, as sorted sphere
 * triples in lexicographic order, keeping those whose longest centre distance
 * is below max_edge (the throat boxes stay bounded).  facets_out: capacity x 3
 * sphere indices (may be NULL when capacity = 0, which only counts).
 * LBM_ERR_ARG as lbm_regular_triangulation, or for a capacity below the count. */
int lbm_packing_throats(const double* spheres, int n, double max_edge, int* facets_out, int capacity,
                        int* n_facets);

/* lbm_pn_build -- the pore network of a lattice sample: pore i is tetrahedron i
 * of tets (n_tets x 4 sphere indices).  Every interior void cell of the mask
 * (mask byte 0: not grain, not a reservoir or membrane layer) belongs to the
 * tetrahedron holding its centre (the lowest index on shared faces); cells
 * outside every tetrahedron join the pore of the nearest such cell through the
 * void (6-neighbour flood).  pore_volume[i] = its cell count.  Throats: every
 * facet shared by two tetrahedra (throat_pores = the two pores, throat_spheres
 * = the facet's three sphere indices), then a link (pore, LBM_PN_INLET) for
 * each pore with a cell next to the inlet layer and (pore, LBM_PN_OUTLET) for
 * each pore with a cell next to the first membrane or outlet layer (spheres
 * -1 -1 -1).  capacity = 0 (arrays may be NULL) only counts into *n_throats.
 *   mask, box  the sample's mask (lbm_get_mask layout) and (nx, ny, nz).
 * LBM_ERR_ARG for bad input or a capacity below the count. */
int lbm_pn_build(const double* spheres, int n_spheres, const int* tets, int n_tets, const unsigned char* mask,
                 const int box[3], double* pore_volume, int* n_throats, int* throat_pores, int* throat_spheres,
                 int capacity);

/* lbm_pn_drainage -- quasi-static primary drainage of a pore network.  Level l
 * imposes capillary pressure p_c[l]; the non-wetting fluid then passes every
 * throat with entry pressure below p_c[l] (strictly) from a non-wetting pore or
 * the non-wetting reservoir into a wetting pore, lowest entry pressure first
 * (ties: lower throat index), until no such throat is left.  A wetting pore
 * without a path of wetting pores to the wetting reservoir is trapped and keeps
 * its fluid ("disconnected regions remain saturated", Sec. 3.1.1); nothing
 * enters the wetting reservoir (membrane).
 *   throat_pores  n_throats x 2: a pore, then a pore or LBM_PN_INLET / _OUTLET.
 *   throat_pce    entry pressures (+inf: never passed).
 *   S_w           n_levels outputs: wetting volume fraction after each level.
 *   pore_invaded_at, pore_trapped_at (n_pores each, may be NULL): the level a
 *                 pore was invaded / trapped at, -1 if never (pores cut off
 *                 from the start are trapped at level 0).
 * LBM_ERR_ARG for bad input. */
int lbm_pn_drainage(int n_pores, const double* pore_volume, int n_throats, const int* throat_pores,
                    const double* throat_pce, int n_levels, const double* p_c, double* S_w,
                    int* pore_invaded_at, int* pore_trapped_at);

/* lbm_partition_lpt -- splits n work items (cost[i] >= 0, e.g. the non-solid
 * cells of a throat box) over `parts` ranks, longest processing time first:
 * items by decreasing cost (ties: lower index), each to the part with the least
 * load so far (ties: lower part).  part_out: n part indices; load_out (may be
 * NULL): the parts' total costs.  Used to shard a throat list over GPUs
 * (Sec. 4: throats are independent, so the only exchange is the final gather
 * of their results). */
int lbm_partition_lpt(const double* cost, int n, int parts, int* part_out, double* load_out);

/* lbm_throat_incircle -- for n throats (n x 3 x (cx, cy, cz, r)), the radius of
 * the throat's inscribed circle: in the plane of the three centres, the largest
 * clearance min_i(|p - c_i| - r_i) over points p of their triangle (the circle
 * touching the three sphere sections when its centre lies in the triangle,
 * else a circle centred on an edge); 0 when the spheres close the throat.
 * r_out: n doubles. */
int lbm_throat_incircle(const double* throats, int n, double* r_out);

/* lbm_throat_pce_incircle -- the incircle estimate of the entry pressure (the
 * approximation Sec. 1 cites): a meniscus of radius r_i / cos(theta) spanning
 * the inscribed circle, p_c^e = 2 sigma cos(theta) / r_i (+inf for a closed
 * throat).  sigma: interfacial tension, cos_theta: of the contact angle. */
int lbm_throat_pce_incircle(const double* throats, int n, double sigma, double cos_theta, double* pce_out);

/* lbm_throat_pce_msp -- the Mayer-Stowe-Princen estimate of the entry pressure
 * (the other approximation Sec. 1 cites), with the throat taken as a prism:
 * its section is the triangle of the three centres minus the sphere sections,
 * its sides neutral walls (90 degrees, as the lattice throat domain's).  At
 * p_c = sigma / r the wetting fluid holds arc menisci of radius r in the
 * corners between grains (meeting the grains at theta, the walls at 90
 * degrees); the non-wetting area A_nw, meniscus length L_nw and grain contact
 * length L_ns of the section then satisfy at entry
 *     p_c^e A_nw = sigma (L_nw + L_ns cos(theta)),
 * solved for r by a scan from 0 in steps of r_i / 64 (r_i the incircle, up to
 * 16 r_i) and bisection; p_c^e = sigma / r.  The non-wetting region is
 * found exactly for any arrangement of the menisci (the part of the section
 * within r of the meniscus centres allowed by the contact angles; its boundary
 * from the arrangement of walls, grain circles and meniscus circles).
 * pce_out[t] = +inf for a closed throat, NaN for collinear centres.
 * cos_theta in (0, 1].  Host, all cores. */
int lbm_throat_pce_msp(const double* throats, int n, double sigma, double cos_theta, double* pce_out);

/* lbm_throat_msp_terms -- the MS-P terms of one throat (3 x (cx, cy, cz, r)) at
 * meniscus radius r: out[0] = A_nw, out[1] = L_nw, out[2] = L_ns (lattice
 * units).  LBM_ERR_ARG for collinear centres, r <= 0 or cos_theta <= 0. */
int lbm_throat_msp_terms(const double* throat, double r, double cos_theta, double out[3]);

/* ---------------------------------------------------------------------------
 * Surrogate network.  The paper reads p_c^e off one LBM run per throat; the
 * surrogate learns that map from LBM-generated throats so that most throats of a
 * large packing need no LBM run, with the LBM as fallback where the ensemble
 * members disagree.  (The paper has no network; this is the build's
 * acceleration of the per-throat step.)  An ensemble of multilayer perceptrons,
 * n_in -> n_layers x n_hidden (ReLU) -> n_out (linear), trained on the mean
 * squared error with Adam.  Every layer runs on the tensor cores with BF16
 * (half = 0) or FP16 (half = 1) operands rounded from FP32 master weights and
 * FP32 accumulation.  Arrays are row-major host float arrays; the parameters of a
 * member are flat: W_0 (out x in), b_0, W_1, b_1, ...
 * ------------------------------------------------------------------------- */
typedef struct lbm_surrogate lbm_surrogate;
typedef struct {
    int n_in, n_hidden, n_layers, n_out;
    int n_members;            /* ensemble size, 1..64                          */
    int half;                 /* 0 = BF16 operands, 1 = FP16 operands          */
    unsigned long long seed;  /* seeded He-normal initialisation per member    */
} lbm_surrogate_config;

int lbm_surrogate_create(const lbm_surrogate_config* cfg, void* stream, lbm_surrogate** out);
int lbm_surrogate_num_params(const lbm_surrogate* s);
int lbm_surrogate_get_params(lbm_surrogate* s, int member, float* params_out);
int lbm_surrogate_set_params(lbm_surrogate* s, int member, const float* params); /* resets its Adam state */
/* lbm_surrogate_forward -- outputs of one member for n inputs (n x n_out). */
int lbm_surrogate_forward(lbm_surrogate* s, int member, const float* X, int n, float* Y);
/* lbm_surrogate_gradients -- gradient of the mean squared error of one member
 * over n samples (flat, parameter layout) and the loss; nothing is updated. */
int lbm_surrogate_gradients(lbm_surrogate* s, int member, const float* X, const float* T, int n, float* grads,
                            double* loss);
/* lbm_surrogate_train -- epochs of minibatch Adam (lr, beta 0.9/0.999) for every
 * member, order shuffled per member and epoch from shuffle_seed; epoch_loss
 * (n_members x epochs, may be NULL) receives the mean batch loss. */
int lbm_surrogate_train(lbm_surrogate* s, const float* X, const float* T, int n, int epochs, int batch, float lr,
                        unsigned long long shuffle_seed, double* epoch_loss);
/* lbm_surrogate_predict -- ensemble mean and standard deviation per output. */
int lbm_surrogate_predict(lbm_surrogate* s, const float* X, int n, float* mean, float* spread);
void lbm_surrogate_destroy(lbm_surrogate* s);
/* lbm_surrogate_selftest_wait -- checks the failure path of the surrogate GEMM's
 * waits for its tensor-core MMAs: one CTA runs the GEMM kernel with the MMA issue
 * switched off, so that its completion barrier never completes, and its bounded
 * waits limited to limit_us microseconds (1 .. 1e7; two waits run out).  *gave_up
 * is set to 1 when the kernel gave up and reported it through its error flag (the
 * expected outcome), 0 otherwise; it frees its tensor memory either way and the
 * context stays usable.  Synchronising (legacy default stream).  No counterpart
 * in the paper. */
int lbm_surrogate_selftest_wait(int limit_us, int* gave_up);

/* ---------------------------------------------------------------------------
 * Throat surrogate: the network above applied to pore throats (no counterpart
 * in the paper, which reads p_c^e off one LBM run per throat, Sec. 2.2.2).
 * Inputs per throat (LBM_SURROGATE_INPUTS): the three radii and the three
 * centre distances over the mean radius R (spheres ordered by decreasing
 * radius, ties in input order) and the contact angle (7); the throat box's
 * lbm_throat_lattice_features (14); their entries 5, 8 and 9 over R (3).
 * Outputs (1 + n_incr): p_c^e R and the throat's S_w after each increment of
 * the training ladder.  Inputs and targets are standardised by the training
 * means and standard deviations (+1e-6).
 * ------------------------------------------------------------------------- */
#define LBM_SURROGATE_INPUTS 24
typedef struct lbm_throat_surrogate lbm_throat_surrogate;
typedef struct {
    int n_incr;               /* increments of the ladder the targets come from      */
    int n_members, n_hidden, n_layers, half;  /* the ensemble (lbm_surrogate_config) */
    unsigned long long seed;  /* initialisation seed                                  */
    double theta;             /* contact angle (radians) in every throat's inputs     */
} lbm_throat_surrogate_config;

/* lbm_contact_angle_estimate -- contact angle of the wall adhesion by the
 * estimate cos(theta) = (G_ads,nw - G_ads,w) / (G (rho_major - rho_minor) / 2)
 * (Huang et al. 2007), clamped to [0, pi]; radians. */
int lbm_contact_angle_estimate(double G_ads_w, double G_ads_nw, double G, double rho_major, double rho_minor,
                               double* theta_out);

/* lbm_pressure_ladder -- per-throat reservoir ladders: n_incr inlet densities
 * per throat (out: n x n_incr, throat-major) whose reservoir capillary pressure
 * p_c,res = (rho_in - rho_major)(1 + G rho_minor)/3 (Eq. 5 on the reservoir
 * layers at rest) runs from lo / r to hi / r in equal steps, r = r_in[i]
 * (floored at 0.5), e.g. the throat's incircle radius. */
int lbm_pressure_ladder(const double* r_in, int n, int n_incr, double lo, double hi, double rho_major,
                        double rho_minor, double G, double* out);

/* lbm_throat_surrogate_inputs -- the inputs of n throats (n x 3 x 4 doubles):
 * X_out n x LBM_SURROGATE_INPUTS floats, R_out (may be NULL) the mean radii. */
int lbm_throat_surrogate_inputs(const double* throats, int n, double theta, float* X_out, double* R_out);

int lbm_throat_surrogate_create(const lbm_throat_surrogate_config* cfg, void* stream, lbm_throat_surrogate** out);

/* lbm_throat_surrogate_fit -- trains on n throats and their batched-LBM outcome
 * (results: n entries, rows: n x n_incr, as lbm_run_throat_batch returns them);
 * throats never invaded within the ladder are left out (*n_used counts the
 * rest).  Sets the standardisation, then lbm_surrogate_train (epochs, batch, lr,
 * shuffle_seed, epoch_loss as there).  LBM_ERR_ARG with fewer than 2 throats. */
int lbm_throat_surrogate_fit(lbm_throat_surrogate* ts, const double* throats, int n, const lbm_throat_result* results,
                             const lbm_increment* rows, int epochs, int batch, float lr, unsigned long long shuffle_seed,
                             double* epoch_loss, int* n_used);

/* lbm_throat_surrogate_predict -- ensemble mean p_c^e (lattice pressure units),
 * its relative spread |std(p_c^e R)| / |mean(p_c^e R)|, and (curves, may be
 * NULL; n x n_incr) the mean S_w curve of n throats.  LBM_ERR_STATE before a fit. */
int lbm_throat_surrogate_predict(lbm_throat_surrogate* ts, const double* throats, int n, double* p_ce,
                                 double* rel_spread, float* curves);

/* lbm_throat_surrogate_predict_with_fallback -- p_c^e of n throats: the
 * ensemble's where its relative spread is at most spread_tol, otherwise the
 * batched LBM's (lbm_run_throat_batch with params and sched on the surrogate's
 * stream; with sched->per_throat the ladders are n x n_incr).  used_lbm[i] = 1
 * for the throats that went to the LBM.  seconds (may be NULL): [network time,
 * LBM time]. */
int lbm_throat_surrogate_predict_with_fallback(lbm_throat_surrogate* ts, const double* throats, int n,
                                               double spread_tol, const lbm_params* params,
                                               const lbm_schedule* sched, double* p_ce, int* used_lbm,
                                               double* seconds);

/* lbm_throat_surrogate_scaling -- the standardisation (LBM_SURROGATE_INPUTS and
 * 1 + n_incr doubles each).  lbm_throat_surrogate_network -- the underlying
 * network (owned by the throat surrogate). */
int lbm_throat_surrogate_scaling(const lbm_throat_surrogate* ts, double* x_mu, double* x_sd, double* y_mu,
                                 double* y_sd);
lbm_surrogate* lbm_throat_surrogate_network(lbm_throat_surrogate* ts);
void lbm_throat_surrogate_destroy(lbm_throat_surrogate* ts);

/* lbm_get_density -- densities of the current state, 2 x N doubles
 * (component-major), 0 where a component is not fluid. Synchronising. */
int lbm_get_density(lbm_domain* d, double* rho_out);

/* lbm_get_mask -- the domain's mask, N bytes. */
int lbm_get_mask(const lbm_domain* d, unsigned char* mask_out);

/* lbm_get_dims -- (nx, ny, nz) and the number of interior fluid cells. */
int lbm_get_dims(const lbm_domain* d, int dims_out[3], long long* n_fluid_cells);

/* lbm_get_state / lbm_set_state -- checkpoint: the stored populations,
 * 2 x 19 x N floats (component, direction, cell), plus the step counter.  The
 * stored values are the post-collision populations of the last step, which the
 * next step pulls from (after lbm_set_densities, values whose pull yields the
 * rest equilibrium).  Resuming from a saved state reproduces the uninterrupted
 * run bit for bit.  FP32 domains only (LBM_ERR_STATE otherwise). */
int lbm_get_state(lbm_domain* d, float* f_out, long long* step_out);
int lbm_set_state(lbm_domain* d, const float* f_in, long long step);

/* lbm_measure_state_noalloc -- the observables of lbm_measure for a state that
 * lives in caller-owned device memory, computed without allocating any device
 * memory.  The paper has no counterpart: this serves callers that must not
 * allocate, such as plug-ins whose host application owns all device memory
 * through its own pool and accounts for every byte, or loops that cannot absorb
 * the device synchronisation of cudaMalloc/cudaFree.
 *   params    model parameters (only G and periodic are read).
 *   box       (nx, ny, nz), each in [1, 4096], at most 56,000,000 cells in all;
 *             larger states are rejected with LBM_ERR_ARG.
 *   f_dev     DEVICE pointer to the stored populations in the lbm_get_state
 *             layout: 2 x 19 x N floats, f[(s*19 + k) * N + cell].
 *   mask_dev  DEVICE pointer to the N mask bytes (layout above); a cell's class
 *             follows the priority solid > inlet > outlet > membrane, as in a
 *             domain created from the same mask.
 *   stream    cudaStream_t to run on (NULL = legacy stream); the call copies its
 *             sums into host memory and waits for the stream before returning.
 *   out       HOST pointer, filled as by lbm_measure.
 * The reduction scratch is a fixed device array inside the library (about
 * 128 KiB, held by every GPU that loads the library until the process exits);
 * each call looks up its device address on the current device (no allocation).
 * All calls share it: calls whose device work overlaps in time race on it.
 * Returns LBM_ERR_NONFINITE like lbm_measure, LBM_ERR_CUDA when a CUDA call
 * fails. */
int lbm_measure_state_noalloc(const lbm_params* params, const int box[3], const float* f_dev,
                              const unsigned char* mask_dev, void* stream, lbm_measurement* out);

/* lbm_set_tile / lbm_get_tile -- launch shape of the fused step kernel.
 *   by    CTA rows including the two halo rows: 6, 8, 10 or 12 (the CTA owns
 *         30 x (by - 2) columns of cells);
 *   lz    planes per CTA z-segment, >= 1;
 *   lead  planes queued ahead of the collided one: 2, 3 or 4 (lead 3 allows
 *         by <= 10, lead 4 allows by <= 8).
 * Results do not depend on the shape (bit for bit).  LBM_ERR_ARG for an
 * unsupported combination (16-bit storage: lead 2 and by 6, 8 or 10). */
int lbm_set_tile(lbm_domain* d, int by, int lz, int lead);
int lbm_get_tile(const lbm_domain* d, int* by, int* lz, int* lead);

/* lbm_set_step_kernel / lbm_get_step_kernel -- which kernel advances an FP32
 * domain (16-bit storage always uses the staged kernel).
 *   LBM_KERNEL_STAGED  every thread queues its cell's 2 x 19 pulls as 4-byte
 *                      asynchronous copies (any box, any periodic axes); its
 *                      shape is set with lbm_set_tile;
 *   LBM_KERNEL_TMA     one thread per CTA loads whole population planes of a
 *                      32 x 8 tile with the tensor memory accelerator (boxes
 *                      without periodic x or y and with nx a multiple of 4);
 *                      lz planes per CTA z-segment (lz <= 0: the default);
 *   LBM_KERNEL_SPLIT   two launches per step: every cell's density pair into a
 *                      field, then pull + collision reading the 18 neighbour
 *                      densities from it (any box; FP32 only; lz ignored);
 *   LBM_KERNEL_STAGED2 the staged kernel with two threads per cell, one per
 *                      fluid component (any box; FP32 only; by 6 or 8, lead 2,
 *                      lz planes per z segment, lz <= 0: keep the current).
 *   LBM_KERNEL_PUSH    the state is kept in a paired push layout (the two
 *                      components of a direction side by side, each cell's
 *                      populations at the current time level at its own
 *                      address, the 19 directions of a row of cells one row
 *                      after another; streaming with bounce-back happens at
 *                      the store); one thread per CTA loads each plane of a
 *                      32-column tile, all 19 directions, with one tensor
 *                      memory accelerator copy (FP32; boxes without periodic x
 *                      or y and with an even nx); lz planes per z segment
 *                      (lz <= 0: keep the current); shape by lbm_set_push_shape.
 *                      Results equal the staged kernel's bit for bit.  The
 *                      state is converted between the layouts when the kind
 *                      changes; lbm_measure, lbm_get_density and
 *                      lbm_get_density_at read the paired layout directly (the
 *                      same bits), lbm_get_state converts a copy into the other
 *                      buffer; callers see the pull layout only.
 *                      On a 16-bit domain the same kind is the 16-bit push
 *                      kernel: each pair word of the pull form is stored at
 *                      the cell that reads it, encoded against the same
 *                      densities; one box load of the words and one of the
 *                      density pairs per plane (boxes without periodic x or y
 *                      and with nx % 4 == 0).  Its results equal the staged
 *                      16-bit kernel's bit for bit; the read-outs convert a
 *                      copy into the pull layout.
 * New domains use LBM_KERNEL_STAGED (lbm_autotune times every kind that applies
 * on the domain).  All give the same results up to rounding (not bit for bit:
 * the TMA kernel folds omega w_k into its equilibrium constants).  LBM_ERR_ARG
 * for an unknown kind, LBM_ERR_STATE when the kernel does not apply to the
 * domain.  lbm_set_tile switches the domain to LBM_KERNEL_STAGED. */
#define LBM_KERNEL_STAGED 0
#define LBM_KERNEL_TMA 1
#define LBM_KERNEL_SPLIT 2
#define LBM_KERNEL_STAGED2 3
#define LBM_KERNEL_PUSH 4
int lbm_set_step_kernel(lbm_domain* d, int kind, int lz);
int lbm_get_step_kernel(const lbm_domain* d, int* kind, int* lz);

/* lbm_set_push_shape -- switches the domain to LBM_KERNEL_PUSH with a CTA shape:
 *   shape  0: 8 box rows (6 interior), 4 plane stages, one CTA per SM;
 *          1: 6 rows, 3 stages, two CTAs per SM; 2: 10 rows, 3 stages, one CTA;
 *          3: 7 rows, 3 stages, two CTAs per SM; 4: 10 rows, 4 stages, one CTA;
 *          5: 12 rows, 3 stages, one CTA;
 *          6 .. 11 keep each cell's populations in registers from the density
 *          pass to the collision, so that every stage holds a load in flight:
 *          6: 6 rows, 3 stages, two CTAs; 7: 10 rows, 4 stages, one CTA;
 *          8: 12 rows, 3 stages, one CTA; 9: 5 rows, 4 stages, two CTAs;
 *          10: 8 rows, 4 stages, one CTA; 11: 7 rows, 3 stages, two CTAs.
 *          A CTA of 32 x rows threads advances 28 x (rows - 2) columns.
 *          On a 16-bit domain (params.precision 1 or 2) the shapes of the
 *          16-bit push kernel: 0: 8 rows, 4 stages; 1: 6 rows, 4 stages;
 *          2: 7 rows, 4 stages; 3: 10 rows, 3 stages; two CTAs per SM each;
 *          6: 9 rows, 3 stages, two CTAs; 7: 7 rows, 3 stages, three CTAs;
 *          8: 6 rows, 3 stages, three CTAs; 9: 11 rows, 3 stages, two CTAs;
 *          4, 5, 10 and 11 keep each cell's pair words in registers from the
 *          density pass to the collision: 4: 6 rows, 4 stages, two CTAs;
 *          5: 8 rows, 4 stages, two CTAs; 10: 12 rows, 3 stages, one CTA;
 *          11: 8 rows, 3 stages, two CTAs.  With tau = 1 in both components a
 *          compile-time tau = 1 form of the collision runs (the same bits).
 *          It needs nx % 4 == 0 (besides no periodic x or y), and its results
 *          equal the staged 16-bit kernel's bit for bit; prefetch and segment
 *          order do not apply to it.
 *   lz     planes per CTA z segment (lz <= 0: a default for the box).
 * Results do not depend on the shape (bit for bit); with tau = 1 in both
 * components a compile-time tau = 1 form of the collision runs (the same bits).
 * LBM_ERR_ARG for an unknown shape, LBM_ERR_STATE when the push kernel does not
 * apply to the domain. */
int lbm_set_push_shape(lbm_domain* d, int shape, int lz);

/* lbm_set_push_prefetch -- how many planes (0 .. 4) the push kernel asks the
 * tensor memory accelerator to bring into L2 beyond the planes whose loads
 * are in flight; a hint that changes no result (bit for bit) and costs no
 * shared memory.  New domains use 0.  Kept across lbm_set_push_shape;
 * lbm_autotune sets it with the shape it picks.  LBM_ERR_ARG outside 0 .. 4. */
int lbm_set_push_prefetch(lbm_domain* d, int planes);

/* lbm_set_push_order -- how the push kernel's CTAs walk the box.  0: tiles in
 * x, y, z-segment launch order, every segment marching towards +z.  1: all z
 * segments of a tile column launched together, alternate segments marching
 * towards -z, so that two neighbouring segments start (or end) at the plane
 * they share at the same time and its halo planes are read from DRAM once.
 * Results do not depend on it (bit for bit).  New domains use 0, and so does
 * lbm_autotune (order 1 was slower in every shape on the drainage sample).
 * LBM_ERR_ARG outside 0 .. 1. */
int lbm_set_push_order(lbm_domain* d, int order);

/* lbm_autotune -- time the step kernels and launch shapes that apply to the
 * domain on the domain itself and keep the fastest.
 *   trial_steps  time steps timed per candidate (>= 1), after one untimed step;
 *   out          optional: the chosen shape and its time per step.
 * Candidates: for FP32 domains the push kernel (where it applies) in every
 * shape with z segments of 16, 24, 32, 48 and 64 planes, each without and
 * with a two-plane L2 prefetch (lbm_set_push_prefetch), in segment order 0
 * (lbm_set_push_order; order 1 is left to the caller), the TMA kernel (where it
 * applies) with z segments of 8 .. 48 planes, the two-launch kernel, the two-threads-per-cell
 * staged kernel (by 6 or 8, z segments of 8 .. 32), and the staged kernel with
 * by in {6, 8, 10}, lead in {0, 1, 2, 3} (0 and 1: the double-pull variant) and
 * z segments of 8 .. 32 planes; for 16-bit storage the staged kernel with by in
 * {6, 8, 10} and lead 2 and (where it applies) the 16-bit push kernel in every
 * shape with z segments of 16, 24, 32 and 48 planes.
 * Timing uses CUDA events on the domain's stream.  The
 * populations, the step counter and (16-bit) the density fields are saved
 * before and restored after, bit for bit: a tuned domain continues exactly where
 * it stood.  Needs one extra population buffer of device memory while it runs
 * (LBM_ERR_OOM otherwise).  Synchronising. */
typedef struct {
    int kind;           /* LBM_KERNEL_* of the chosen kernel */
    int by, lz, lead;   /* the shape: staged kernels by and lead; push kernel box
                           rows (by) and plane stages (lead); lz the z segment */
    double ms_per_step; /* its measured time per step */
    int n_candidates;   /* shapes timed */
    int prefetch;       /* push kernel: its L2 prefetch distance in planes; else 0 */
    int shape;          /* push kernel: its lbm_set_push_shape index; else -1 */
    int order;          /* push kernel: its lbm_set_push_order; else 0 */
} lbm_tune_result;
int lbm_autotune(lbm_domain* d, int trial_steps, lbm_tune_result* out);

/* lbm_selftest_bounded_wait -- checks the failure path of the TMA step kernel's
 * waits on the GPU: one CTA waits on an mbarrier that nothing ever completes,
 * with the same bounded wait the kernel uses, limited to limit_us microseconds
 * (1 .. 1e7).  *gave_up is set to 1 when the wait gave up and reported it (the
 * expected outcome), 0 otherwise.  No copy is in flight and the context stays
 * usable.  Synchronising (legacy default stream).  No counterpart in the paper. */
int lbm_selftest_bounded_wait(int limit_us, int* gave_up);

/* lbm_destroy -- release the domain (NULL is ignored). */
void lbm_destroy(lbm_domain* d);

/* lbm_last_error -- description of the last failure on this thread. */
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H_ */
