/*
 * slh.h -- C ABI of the GB300 AMR axion-string stepper.
 *
 * The library advances the complex scalar psi = psi1 + i psi2 and its momenta
 * Pi1, Pi2 of arXiv:2404.02950 (sledgehamr) Sec. 3.1 on a block-structured
 * hierarchy of periodic levels (Sec. 2): ghost-padded boxes, refinement
 * ratio 2, dt_l = dt_0 / 2^l (Eqs. 1-3), recursive time subcycling with
 * spatial + temporal ghost interpolation and fine-to-coarse averaging at
 * synchronisation (Sec. 2.1, Fig. 2), classic RK4 (integrator type 4 of the
 * "integrator" table), string-winding refinement tags (the problem-specific
 * tagging hook of Sec. 4.2) and Berger-Rigoutsos style regridding
 * (Sec. 2.2-2.3).  Optionally (nfields = 16) it also evolves the auxiliary
 * gravitational-wave tensor of Sec. 5: six components u_ij (xx, yy, zz, xy,
 * xz, yz) and their conformal-time derivatives v_ij, with
 *   u_ij' = v_ij
 *   v_ij' = -c_fric v_ij + lap u_ij + 2 (d_i psi1 d_j psi1 + d_i psi2 d_j psi2)
 * (the string-network source of Eq. GWEOM in conformal time; the gradients
 * are the central differences of accuracy lap_order, App. A).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Status: every function returns slh_status; 0 is success, negative values
 *    are the SLH_ERR_* codes below.  slh_last_error() returns a thread-local
 *    message describing the last failure.  No C++ exception crosses the ABI.
 *  - Device-side failures (a bounded wait that gave up, a consistency check
 *    inside a kernel) are latched in a device word; the next synchronising
 *    call (slh_sync, slh_reduce_energy, slh_tag, slh_get_state to host)
 *    returns them.  Kernels never trap.
 *  - Streams: every call that launches work is asynchronous on the stream
 *    given to slh_create (a cudaStream_t passed as void*), except where noted.
 *  - Ownership: field buffers are allocated by the caller (e.g. PyTorch) and
 *    passed as device pointers; the library never frees them and never
 *    retains them past slh_init_level of the same level or slh_destroy.
 *    The library owns only metadata (box tables, block maps, work lists,
 *    reduction partials, CUDA graphs), released by slh_destroy.
 *  - Layout: arrays are x fastest, then y, then z.  A box (slh_box) holds
 *    inclusive lo/hi cell indices in its level's index space; boxes of a
 *    level are disjoint, multiples of and aligned to the blocking factor.
 *    In device buffers each box is stored component by component
 *    (psi1, psi2, Pi1, Pi2, then with 16 fields u_xx, u_yy, u_zz, u_xy, u_xz,
 *    u_yz, v_xx, ..., v_yz) with nghost ghost layers in y and z and a
 *    16-byte aligned x padding; slh_level_layout reports the offsets.
 *    "Dense" host/device arrays (slh_set_state / slh_get_state, tags) hold
 *    only valid cells: [box][component][z][y][x] with boxes in list order.
 */
#ifndef SLH_H
#define SLH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t slh_status;

#define SLH_OK 0
#define SLH_ERR_INVALID_ARG (-1)  /* null pointer, bad enum, inconsistent sizes */
#define SLH_ERR_OUT_OF_RANGE (-2) /* box outside the domain, level index, capacity */
#define SLH_ERR_CUDA (-3)         /* a CUDA runtime call failed */
#define SLH_ERR_TIMEOUT (-4)      /* a bounded device wait gave up */
#define SLH_ERR_NOMEM (-5)        /* metadata allocation failed */
#define SLH_ERR_DEVICE (-6)       /* a device-side consistency check failed */
#define SLH_ERR_STATE (-7)        /* call out of order (level not initialised ...) */

/* Storage / arithmetic precision of the fields. */
#define SLH_F64 0        /* FP64 fields, FP64 arithmetic */
#define SLH_F32_KAHAN 2  /* FP32 fields and arithmetic, Kahan-compensated final
                            RK update; FP64 only for eta, its coefficients and
                            the reductions */
#define SLH_F32_BF16 3   /* 16 fields: psi, Pi in FP32, the tensor fields u_ij,
                            v_ij stored in BF16 (rounded to nearest even),
                            FP32 arithmetic and accumulation; a cell holds 10
                            slots of 4 bytes (SLH_SLOTS_BF16); three level
                            buffers (SLH_BUF_Y, YA, YB; D and C stay NULL);
                            integrator SSPRK3 (type 10 or 3) only */
#define SLH_SLOTS_BF16 10 /* slots of an SLH_F32_BF16 cell: psi1, psi2, Pi1, Pi2
                            in FP32, then the BF16 pairs (u_xx, u_yy),
                            (u_zz, u_xy), (u_xz, u_yz), (v_xx, v_yy),
                            (v_zz, v_xy), (v_xz, v_yz), the first of each pair
                            in the low 16 bits */

/* Buffers of one level (device pointers handed to slh_init_level). */
#define SLH_BUF_Y 0      /* state y_n (rotates with SLH_BUF_YB every step) */
#define SLH_BUF_YA 1     /* RK stage value */
#define SLH_BUF_YB 2     /* RK stage value / the level's previous state */
#define SLH_BUF_D 3      /* RK increment accumulator */
#define SLH_BUF_C 4      /* Kahan compensation (SLH_F32_KAHAN only, else NULL) */
#define SLH_NBUF 5

/* slh_rk_step / slh_advance flags */
#define SLH_FUSE_TAG 1u     /* stage 1 also writes the winding tags of y_n */
#define SLH_FUSE_ENERGY 2u  /* stage 1 also accumulates the energy of y_n */
#define SLH_USE_GRAPH 4u    /* slh_advance: replay a captured CUDA graph */

/* Refinement criteria (slh_set_tagging); the block mask of slh_tag_blocks
 * is the union of the enabled ones */
#define SLH_TAG_WINDING 1u  /* string winding (the problem-specific hook of Sec. 4.2) */
#define SLH_TAG_TEE 2u      /* truncation-error estimate (Sec. 2.2) */

/* slh_fill_ghosts modes */
#define SLH_GHOSTS 0     /* fill the psi (and u_ij) ghosts of the level's state */
#define SLH_RESTRICT 1   /* average the level onto the next coarser one
                            (covered cells, every field), then refill
                            this level's psi (and u_ij) ghosts */

/* Profiling counters (slh_profile_read kinds) */
#define SLH_PROF_STAGE 0     /* all four RK stages (sum of SLH_PROF_S1..S4) */
#define SLH_PROF_GHOST 1
#define SLH_PROF_RESTRICT 2
#define SLH_PROF_DIAG 3
#define SLH_PROF_TIME 4
#define SLH_PROF_S1 5        /* RK stage 1 .. 4 separately */
#define SLH_PROF_S2 6
#define SLH_PROF_S3 7
#define SLH_PROF_S4 8
#define SLH_PROF_GW 9        /* the gravitational-wave stage kernel (16 fields) */
#define SLH_PROF_KO 10       /* the dissipation kernel */
/* host wall-clock phases, recorded whether or not profiling is enabled
 * (cleared by slh_profile's reset): */
#define SLH_PROF_REGRID_TAGS 11     /* slh_regrid: tags and block masks (device + copy back) */
#define SLH_PROF_REGRID_CLUSTER 12  /* slh_regrid: host clustering (global or local) */
#define SLH_PROF_REGRID_BUILD 13    /* slh_regrid: caller's allocator + level rebuild */
#define SLH_PROF_GRAPH_CAPTURE 14   /* slh_advance: capture and instantiation of a graph */
#define SLH_PROF_NKINDS 15

typedef struct {
  int32_t lo[3];
  int32_t hi[3];
} slh_box;

/* Coefficients of the equations of motion (Sec. 3.1, Eqs. EOM1-EOM2):
 *   psi_i' = Pi_i
 *   Pi_i'  = -c_fric Pi_i + lap psi_i - psi_i (c_pot (psi1^2+psi2^2-1) + a)
 * with c_fric = 2/eta (friction = 1) or 0, c_pot = lambda eta^eta_power
 * (eta_power 2 as in the paper, 0 freezes it), the Laplacian of accuracy
 * lap_order in {2,4,6} (the 7/13/19-point stencils of App. A, ghost width
 * lap_order/2), and ghost prolongation interp_type in {0,2,4} (the
 * "interpolation_type" entry of the "amr" table; 4 = quartic conservative;
 * type 1, linear conservative, is not built and returns INVALID_ARG). */
typedef struct {
  double lambda;
  double a;
  int32_t friction;
  int32_t eta_power;
  int32_t lap_order;
  int32_t interp_type;
  int32_t integrator;   /* Tab. "integrator" type: 4 = classic RK4; 10 (or 3) =
                           low-storage SSPRK3, Shu-Osher form: stages at
                           c = (0, 1, 1/2), out = a_s y_n + b_s (Y_s + dt k_s),
                           (a, b) = (0, 1), (3/4, 1/4), (1/3, 2/3); 21 = RKN4,
                           Nystrom's fourth-order method for x'' = a(t, x, x')
                           with positions psi (u_ij), velocities Pi (v_ij):
                           a1 at (x, v); a2 at (x + dt/2 v + dt^2/8 a1,
                           v + dt/2 a1); a3 at (same x, v + dt/2 a2); a4 at
                           (x + dt v + dt^2/2 a3, v + dt a3), stages at
                           c = (0, 1/2, 1/2, 1); x' = x + dt v + dt^2/6 (a1 +
                           a2 + a3), v' = v + dt/6 (a1 + 2 a2 + 2 a3 + a4).
                           RKN4 takes no Kreiss-Oliger term (it needs x' = v).
                           22 = RKN5, Nystrom's fifth-order method for
                           x'' = a(t, x) (friction must be 0; scalar fields
                           only): stages at c = (0, 1/5, 2/3, 1), a_s at
                           x + c_s dt v + dt^2 sum_j abar_sj a_j with abar rows
                           (1/50), (-1/27, 7/27), (3/10, -2/35, 9/35);
                           x' = x + dt v + dt^2 (14 a1 + 100 a2 + 54 a3)/336,
                           v' = v + dt (14 a1 + 125 a2 + 162 a3 + 35 a4)/336;
                           no Kreiss-Oliger term either */
  int32_t pad_;
  double ko_eps;        /* Kreiss-Oliger dissipation (Sec. 2.4) added to the
                           evolution of psi1, psi2, Pi1, Pi2:
                           (-1)^((p+3)/2) eps dx^p / 2^(p+1) sum_d d^(p+1)/dx_d^(p+1)
                           with the central (p+2)-point difference; strength eps */
  int32_t ko_order;     /* p in {1, 3, 5}, 0 = off; needs nghost >= (p+1)/2 */
  int32_t pad2_;
} slh_eom_params;

typedef struct slh_ctx slh_ctx;

/* Message of the last failure on this thread ("" if none). */
const char* slh_last_error(void);

/* Create a hierarchy whose level 0 spans n0^3 cells of spacing dx0 on a
 * periodic domain.  nghost in [1,4] ghost layers (>= lap_order/2, and >= 2
 * for quartic prolongation), blocking_factor a power of two >= 2 dividing
 * n0, prec SLH_F64 or SLH_F32_KAHAN, max_levels in [1,8], nfields 4 (the
 * scalar field and momenta) or 16 (plus the gravitational-wave tensor u_ij,
 * v_ij), stream a cudaStream_t (NULL = legacy default stream).  Allocates
 * metadata only.  Errors: INVALID_ARG, NOMEM, CUDA. */
slh_status slh_create(slh_ctx** ctx, int32_t n0, double dx0, int32_t nghost,
                      int32_t blocking_factor, int32_t prec, int32_t max_levels,
                      int32_t nfields, void* stream);

/* Release the metadata of ctx (field buffers stay with the caller). */
void slh_destroy(slh_ctx* ctx);

/* Element counts of one level buffer of nfields (4 or 16) fields, or of
 * SLH_SLOTS_BF16 slots (a 16-field SLH_F32_BF16 level: elements of 4 bytes),
 * for the given boxes, without a context.  box_offsets (nboxes entries, may be NULL) receives each box's
 * element offset; box_geom (4*nboxes, may be NULL) receives pitch (x row
 * length incl. padding), padded ny, padded nz and the component stride in
 * elements.  The valid cell (x,y,z) of box b, component c, sits at
 *   off_b + c*cstride_b + ((z-lo_z+nghost)*pny_b + (y-lo_y+nghost))*pitch_b
 *         + (x-lo_x+4).
 * *total_elems receives the buffer length in elements; *nvalid the number
 * of valid cells over all boxes.  Errors: INVALID_ARG. */
slh_status slh_level_layout(int32_t nghost, int32_t nfields, const slh_box* boxes, int32_t nboxes,
                            int64_t* box_offsets, int64_t* box_geom,
                            int64_t* total_elems, int64_t* nvalid);

/* Define level lev (0 <= lev < max_levels; levels are defined in order,
 * redefining a level drops the finer ones) with its boxes in the level's
 * index space (domain n0*2^lev).  bufs[SLH_NBUF] are caller-owned device
 * buffers of total_elems elements of the context precision (bufs[SLH_BUF_C]
 * NULL unless SLH_F32_KAHAN); tags_dev, if not NULL, holds nvalid bytes for
 * fused tags.  Level 0 must cover the domain; level lev>0 must lie inside
 * level lev-1 with a gap of at least one block of blocking_factor/2 cells of
 * lev-1 (nesting, Sec. 2.1).  Ghost cells and the Kahan buffer are zeroed.
 * Errors: INVALID_ARG, OUT_OF_RANGE, NOMEM, CUDA. */
slh_status slh_init_level(slh_ctx* ctx, int32_t lev, const slh_box* boxes, int32_t nboxes,
                          void* const* bufs, uint8_t* tags_dev);

/* Global regrid of a live level (Sec. 2.3): give level lev (1 <= lev <=
 * number of levels; lev equal to it creates a new finest level) the boxes
 * boxes[nboxes] with caller-owned buffers bufs[SLH_NBUF] laid out as for
 * slh_init_level.  Every valid cell of the new boxes takes the old level's
 * value where an old box covers it, otherwise the ratio-2 prolongation
 * (interp_type 0/2/4) of level lev-1's current state, every field; the
 * Kahan compensation is carried over where covered and zero elsewhere.  The
 * new level's previous state equals its state and its eta that of lev-1.
 * A level that existed keeps its tile variants (slh_set_tile,
 * slh_set_diag_tile, the autotuners); a new one starts on variant 0.
 * nboxes == 0 removes level lev and every finer level.  Finer levels keep
 * their data but must be regridded (from the new lev) before the next
 * slh_rk_step / slh_advance (SLH_ERR_STATE otherwise).  Regrid coarse to
 * fine, at a synchronised time (after slh_advance).  The old buffers of lev
 * are no longer referenced when the call returns (it synchronises).
 * Errors: INVALID_ARG, OUT_OF_RANGE (nesting), STATE, NOMEM, CUDA. */
slh_status slh_regrid_level(slh_ctx* ctx, int32_t lev, const slh_box* boxes, int32_t nboxes,
                            void* const* bufs, uint8_t* tags_dev, int32_t interp_type);

/* Copy the fields (4 or 16) of level lev from / to a dense valid-cell array
 * ([box][comp][z][y][x], context precision; for SLH_F32_BF16 the 10 slots
 * of 4 bytes, [box][slot][z][y][x]).  src/dst on the host
 * (is_host = 1, ideally pinned) or the device.  slh_set_state also sets the
 * level's previous state equal to it and zeroes the Kahan compensation.
 * slh_get_state to host synchronises.  Errors: INVALID_ARG, STATE, CUDA. */
slh_status slh_set_state(slh_ctx* ctx, int32_t lev, const void* src, int32_t src_is_host);
slh_status slh_get_state(slh_ctx* ctx, int32_t lev, void* dst, int32_t dst_is_host);

/* Which of the level's buffers (SLH_BUF_*) currently hold its state,
 * its previous state and the stage scratch: roles[0..2].  Classic RK4 and
 * the Nystrom methods swap the first two every step; SSPRK3 rotates all
 * three (state <- scratch, previous <- state, scratch <- previous).
 * Errors: INVALID_ARG, STATE. */
slh_status slh_level_roles(slh_ctx* ctx, int32_t lev, int32_t roles[3]);

/* Set the conformal time eta of every level (kept in FP64 on the device). */
slh_status slh_set_eta(slh_ctx* ctx, double eta);
/* Read eta of level lev (synchronises). */
slh_status slh_get_eta(slh_ctx* ctx, int32_t lev, double* eta);

/* One step of the integrator p->integrator (classic RK4, SSPRK3, RKN4 or RKN5) of level lev by
 * dt_lev = dt0 / 2^lev.  For lev > 0, sub in {0,1} is the sub-step within
 * the coarser level's step: the level starts at eta_coarse_start +
 * sub*dt_lev and each stage fills psi (and u_ij) ghosts from the coarser level at time
 * fraction (sub + c_s)/2, with the integrator's stage times c (Sec. 2.1).  Before each
 * stage the ghost fill of level lev runs; the four fused stage kernels then
 * compute the RHS of Sec. 3.1 with the stage-time coefficients (with 16
 * fields a second kernel per stage advances u_ij, v_ij the same way).  flags:
 * SLH_FUSE_TAG (tags of y_n into the level's tags_dev), SLH_FUSE_ENERGY
 * (energy partials of y_n, read with slh_reduce_energy mode 1).
 * Errors: INVALID_ARG, STATE, CUDA. */
slh_status slh_rk_step(slh_ctx* ctx, int32_t lev, int32_t sub, double dt0,
                       const slh_eom_params* p, uint32_t flags);

/* One coarse step of the whole hierarchy: the Berger-Oliger recursion of
 * Sec. 2.1 / Fig. 2 (level l one step, level l+1 twice, then
 * SLH_RESTRICT of l+1 onto l).  flags as slh_rk_step plus SLH_USE_GRAPH
 * (capture the step into a CUDA graph on first use and replay it; the
 * graph is rebuilt when a level or the parameters change).
 * Errors: INVALID_ARG, STATE, CUDA. */
slh_status slh_advance(slh_ctx* ctx, double dt0, const slh_eom_params* p, uint32_t flags);

/* Ghost fill / synchronisation of level lev (Sec. 2.1).  mode SLH_GHOSTS:
 * psi (and u_ij) ghosts of the level's state from its own boxes (periodic wrap) and,
 * where uncovered, by ratio-2 prolongation (interp_type 0/2/4) of the
 * coarser level interpolated in time at fraction alpha in [0,1] between its
 * previous and current state.  mode SLH_RESTRICT (lev >= 1): every cell of
 * lev-1 covered by lev becomes the mean of its 8 children (sums in FP64),
 * then lev's ghosts are refilled at alpha = 1.  Errors: INVALID_ARG, STATE,
 * CUDA. */
slh_status slh_fill_ghosts(slh_ctx* ctx, int32_t lev, double alpha, int32_t interp_type,
                           int32_t mode);

/* String-winding tags of level lev's state (rule: a cell is tagged when one
 * of the 12 plaquettes it is a corner of has nonzero winding; plaquette
 * winding counted from the signs of Im psi and of the cross products of
 * neighbouring corners, in FP64).  Ghosts are filled first (alpha = 1).
 * tags_dev: nvalid bytes (dense valid-cell layout) written 0/1.
 * *n_tagged_host (may be NULL) receives the count (synchronises).
 * Errors: INVALID_ARG, STATE, CUDA, and latched device errors. */
slh_status slh_tag(slh_ctx* ctx, int32_t lev, uint8_t* tags_dev, int64_t* n_tagged_host);

/* Block mask for regridding from level lev: the tags of lev (the union of
 * the criteria enabled by slh_set_tagging: winding tags computed now, and
 * the level's last TEE tags), grown by n_error_buf cells (cube, periodic,
 * across boxes), coarsened to blocks of blocking_factor/2 cells:
 * mask_host[(bz*nb + by)*nb + bx] = 1 when the grown tag set meets block
 * (bx,by,bz), nb = (n0*2^lev)/(blocking_factor/2).
 * Synchronises.  Errors: INVALID_ARG, STATE, CUDA. */
slh_status slh_tag_blocks(slh_ctx* ctx, int32_t lev, int32_t n_error_buf, uint8_t* mask_host);

/* Refinement criteria (Sec. 2.2): criteria is a nonzero combination of
 * SLH_TAG_WINDING and SLH_TAG_TEE (default: SLH_TAG_WINDING).  With
 * SLH_TAG_TEE, te_crit[4] are the thresholds eps of (psi1, psi2, Pi1, Pi2)
 * (a threshold <= 0 leaves its component out); the library keeps one tag
 * byte per valid cell of every level (allocated here and whenever a level
 * is defined) and fills it with the truncation-error estimate
 *   Delta phi_cf = |phi_coarse - phi_fine|:
 *  - level l >= 1, at every synchronisation of l with l-1 (SLH_RESTRICT,
 *    including the ones inside slh_advance): the coarse values of l-1 just
 *    before they are replaced against the mean of their 8 children (the
 *    self-shadow method; FP64 comparison);
 *  - level 0, from a shadow context: slh_shadow_init / slh_shadow_compare.
 * A fine cell is tagged when its parent's estimate exceeds eps for some
 * component.  Synchronises.  Errors: INVALID_ARG, NOMEM, CUDA. */
slh_status slh_set_tagging(slh_ctx* ctx, uint32_t criteria, const double* te_crit);

/* Shadow level of level 0 (Sec. 2.2): shadow is a context of the same
 * precision and field count with n0/2 cells of spacing 2 dx0 and its level
 * 0 defined.  slh_shadow_init writes the 2^3 mean of ctx's level 0 (every
 * field) into the shadow's state (its previous state too, Kahan zeroed) and
 * gives it ctx's eta.  Advance the shadow by one step of 2 dt0
 * (slh_rk_step) while ctx advances two coarse steps, then slh_shadow_compare
 * writes level 0's TEE tags from |shadow - mean of children|.  Both order
 * the work of the two streams with events.
 * Errors: INVALID_ARG, STATE, CUDA. */
slh_status slh_shadow_init(slh_ctx* ctx, slh_ctx* shadow);
slh_status slh_shadow_compare(slh_ctx* ctx, slh_ctx* shadow);

/* Gravitational-wave spectrum of level 0 (Sec. 7.4, Eq. gw_spectrum; needs
 * nfields 16): G(n^2) = N^-6 sum over the modes k with |n(k)|^2 = n^2 of
 * Lambda_ij,lm(k) v~_ij(k) v~*_lm(k), v~ the unnormalised DFT of v_ij = u_ij'
 * over the N^3 cells of level 0, n(k) the signed integer frequencies,
 * Lambda_ij,lm = P_il P_jm - P_ij P_lm / 2 with P = 1 - khat khat (Sec. 5,
 * Eq. Lambda_ijlm) and khat the unit effective lattice momentum of
 * projection type ptype: 1, k_eff = sin(theta)/dx (second-order gradients),
 * or 2, k_eff = (8 sin(theta) - sin(2 theta))/(6 dx) (fourth order), theta =
 * 2 pi n/N per axis; khat = 0 where k_eff vanishes.  Writes the distinct n^2
 * values that occur, ascending, to n2_out and the spectrum to g_out (host
 * arrays of capacity cap); *nout receives the number of entries (with
 * OUT_OF_RANGE if cap is smaller).  Uses cuFFT, loaded on first use, and
 * device scratch of about 12 N^3 field values for the call.  Synchronises.
 * Errors: INVALID_ARG, STATE, OUT_OF_RANGE, NOMEM, CUDA. */
slh_status slh_gw_spectrum(slh_ctx* ctx, int32_t ptype, int64_t* n2_out, double* g_out, int32_t cap,
                           int32_t* nout);

/* Copy level lev's TEE tags (nvalid bytes, dense valid-cell layout) to dst
 * (host if dst_is_host, which synchronises, else device).
 * Errors: INVALID_ARG, STATE (TEE not enabled), CUDA. */
slh_status slh_tee_tags(slh_ctx* ctx, int32_t lev, uint8_t* dst, int32_t dst_is_host);

/* Host-only, deterministic regrid: dense tags over a level's whole index
 * domain dims[3] (x,y,z; uint8, x fastest) -> boxes of the next finer level
 * (Sec. 2.2-2.3): grow tags by n_error_buf (cube, periodic), coarsen to
 * blocks of blocking_factor/2 cells, keep blocks inside the parent boxes
 * eroded by one block (parent NULL / nparent 0: the periodic domain), and
 * cluster Berger-Rigoutsos style: accept a box when 10*tags >= 7*volume,
 * sides <= max_box fine cells and inside the allowed blocks; else cut at the
 * zero-signature plane nearest the centre, else at the strongest sign change
 * of the signature's second difference, else halve the longest side (ties:
 * lowest axis x<y<z, then lowest plane).  Output boxes are in the finer
 * level's cells, sorted by (lo_z, lo_y, lo_x).  cap = capacity of out.
 * Errors: INVALID_ARG, OUT_OF_RANGE (cap too small; *nout = needed). */
slh_status slh_regrid_boxes(const uint8_t* tags_host, const int32_t dims[3],
                            int32_t blocking_factor, int32_t n_error_buf, int32_t max_box,
                            const slh_box* parent, int32_t nparent, slh_box* out, int32_t cap,
                            int32_t* nout);

/* Host-only local regrid (Sec. 2.3): keep every level's boxes and only add.
 * boxes: the current boxes of levels 0..nlevels-1, concatenated (nboxes[l]
 * per level; level 0 covers the domain of n0 cells); masks[l] (l < nlevels-1,
 * NULL = no tags): the block mask of level l as slh_tag_blocks returns it
 * (grown tags in blocks of blocking_factor/2 cells of l, x fastest).
 * Steps: a block of masks[l] not covered by level l+1 becomes a new block of
 * blocking_factor cells of level l+1; then, finest level first, every block
 * of level j needs the 3x3x3 blocks of blocking_factor/2 cells of level j-1
 * around it (periodic) inside level j-1, and the missing blocks of
 * blocking_factor cells are added to level j-1 (level 0 never changes).
 * out receives each level's old boxes in their order followed by its new
 * blocks merged into x-runs (ordered by z, y, x), levels concatenated;
 * out_nboxes[l] the count per level.  cap = capacity of out (entries).
 * Errors: INVALID_ARG, OUT_OF_RANGE (cap too small; out_nboxes filled). */
slh_status slh_local_regrid_boxes(int32_t nlevels, int32_t n0, int32_t blocking_factor,
                                  const uint8_t* const* masks, const slh_box* boxes,
                                  const int32_t* nboxes, slh_box* out, int32_t cap,
                                  int32_t* out_nboxes);

/* slh_regrid modes */
#define SLH_REGRID_GLOBAL 0  /* cluster the grown tags of every level anew */
#define SLH_REGRID_LOCAL 1   /* keep every box, only add where needed */
#define SLH_REGRID_AUTO 2    /* local, with the fallback rule below */

/* Parameters of slh_regrid (Sec. 2.2-2.3 and the "amr" table of App. F). */
typedef struct {
  int32_t mode;          /* SLH_REGRID_GLOBAL, SLH_REGRID_LOCAL or SLH_REGRID_AUTO */
  int32_t max_levels;    /* levels the hierarchy may hold afterwards, in [1, ctx max_levels] */
  int32_t start;         /* global: levels <= start keep their boxes; the tags of level start
                            give level start+1 (0: regrid every level above the base) */
  int32_t n_error_buf;   /* cells the tags are grown by ("n_error_buf") */
  int32_t max_box;       /* largest box side in cells of the new level, a multiple of the
                            blocking factor */
  int32_t interp_type;   /* prolongation of new cells: 0, 2 or 4 */
  int32_t max_local;     /* auto: local regrids in a row after which a global one runs
                            ("max_local_regrids", paper default 10; 0 = no cap) */
  int32_t pad_;
  double eps_strong;     /* auto: added-volume fraction that forces a global regrid
                            ("volume_threshold_strong" - 1, paper default 0.1) */
  double eps_weak;       /* auto: fraction from which a level is regridded with it
                            ("volume_threshold_weak" - 1, paper default 0.05) */
} slh_regrid_params;

/* Caller's allocator for the levels slh_regrid rebuilds.  Called with the
 * new boxes of level lev, the buffer length total_elems (elements of the
 * context precision, as slh_level_layout) and nvalid; it stores SLH_NBUF
 * device pointers in bufs (bufs[SLH_BUF_C] may stay NULL unless
 * SLH_F32_KAHAN) and, optionally, a device buffer of nvalid bytes for fused
 * tags in *tags_dev (left NULL: none).  The buffers must stay valid while
 * the level exists; the level's previous buffers are no longer referenced
 * once the rebuild of lev returns.  Called with nboxes = 0 (boxes, bufs,
 * tags_dev NULL) after level lev and every finer level were removed.
 * Returns 0 on success, nonzero to abort the regrid (SLH_ERR_NOMEM). */
typedef int32_t (*slh_level_alloc_fn)(void* user, int32_t lev, const slh_box* boxes, int32_t nboxes,
                                      int64_t total_elems, int64_t nvalid, void** bufs, uint8_t** tags_dev);

/* Regrid the live hierarchy at a synchronised time (after slh_advance),
 * Sec. 2.2-2.3.
 *  - Global: for l = start, start+1, ...: the block mask of level l
 *    (slh_tag_blocks: the enabled criteria, grown by n_error_buf, in blocks
 *    of blocking_factor/2 cells), clustered as slh_regrid_boxes does inside
 *    level l's boxes eroded by one block (l > 0), gives the boxes of level
 *    l+1 (at most max_levels levels), which is rebuilt (slh_regrid_level)
 *    before its own tags give level l+2; an empty list removes the level and
 *    every finer one.
 *  - Local: the block masks of every level but the finest, then
 *    slh_local_regrid_boxes; the levels from the lowest one that gained
 *    cells upward are rebuilt.
 *  - Auto (the paper's fallback rule): the volume local regrids added to
 *    each level since the last global regrid is tracked as a fraction dV_l
 *    of the level's volume then.  The regrid is global when the hierarchy
 *    has fewer than max_levels levels, or when the previous local regrid
 *    left dV_l >= eps_strong on some level or was the max_local-th in a row:
 *    it then starts from level l0 - 1, l0 the lowest level >= 1 with
 *    dV_l >= eps_weak (level 0 if none).  Otherwise it is local.  A global
 *    regrid restarts the counts from the new volumes.
 * Levels are rebuilt with buffers from alloc(user, ...).  *kind (may be
 * NULL) receives SLH_REGRID_GLOBAL or SLH_REGRID_LOCAL; frac (may be NULL,
 * one entry per level before the call) receives dV_l after an auto local
 * regrid, or the cells each level gained in mode local.  Synchronises.
 * Errors: INVALID_ARG, STATE, NOMEM, CUDA; a failure part way leaves the
 * levels rebuilt so far in place. */
slh_status slh_regrid(slh_ctx* ctx, const slh_regrid_params* rp, slh_level_alloc_fn alloc, void* user,
                      int32_t* kind, double* frac);

/* Energy and string length of the hierarchy over the cells not covered by
 * a finer level, each level at its own eta:
 *   out[0] = sum 1/2 (Pi1^2 + Pi2^2) dx^3
 *   out[1] = sum -1/2 (psi1 L psi1 + psi2 L psi2) dx^3   (L = FD Laplacian)
 *   out[2] = sum [c_pot/4 (|psi|^2-1)^2 + a/2 |psi|^2] dx^3
 *   out[3] = out[0] + out[1] + out[2]
 *   out[4] = (number of plaquettes with nonzero winding) dx
 * mode 0: compute now (fills ghosts at alpha = 1 first).  mode 1: return the
 * partials fused into the last SLH_FUSE_ENERGY stage 1 (energy of the state
 * at the start of that step; single level only).  FP64 accumulation in a
 * fixed order (bit-reproducible).  Synchronises.
 * Errors: INVALID_ARG, STATE, CUDA, and latched device errors. */
slh_status slh_reduce_energy(slh_ctx* ctx, const slh_eom_params* p, int32_t mode, double out[5]);

/* Stage-kernel tile shape of level lev: variant indexes a fixed table of
 * (x extent, y extent, TMA pipeline depth, z-march length) shapes; 0 is the
 * default.  FP32 forms: 32x16/2/64, 32x8/3/64, 32x16/3/128, 16x16/2/64,
 * 64x8/2/64, 32x8/3/128, 128x4/2/64 (7 variants); FP64: 32x8/2/64,
 * 32x4/3/64, 16x8/2/64 (3).  The autotuners' ms_out needs one entry per
 * variant (8 always suffice).  Sets the tile of every stage, the diagnostics
 * stage 1 (fused tags and energy) included.  Synchronises.
 * Errors: INVALID_ARG, STATE, OUT_OF_RANGE. */
slh_status slh_set_tile(slh_ctx* ctx, int32_t lev, int32_t variant);

/* As slh_set_tile, for the diagnostics stage only: the stage-1 launch that
 * fuses the winding tags and/or the energy partials (SLH_FUSE_TAG,
 * SLH_FUSE_ENERGY) and the diagnostics pass of slh_tag and of
 * slh_reduce_energy mode 0.  The other stages keep their tile.
 * Synchronises.  Errors: INVALID_ARG, STATE, OUT_OF_RANGE. */
slh_status slh_set_diag_tile(slh_ctx* ctx, int32_t lev, int32_t variant);

/* Autotuner: time every tile variant on level lev's own boxes (reps
 * launches of a middle RK stage in the form p->integrator runs it -- stage 2
 * of classic RK4 or SSPRK3, stage 3 of RKN4 or RKN5 -- that reads the state,
 * SLH_BUF_YA and SLH_BUF_D and writes only the scratch buffers SLH_BUF_YA and
 * SLH_BUF_D), keep the fastest.  *chosen receives its
 * index, ms_out (may be NULL, one entry per variant) the mean milliseconds.
 * Call between steps, outside stream capture.  Synchronises.
 * Errors: INVALID_ARG, STATE, CUDA. */
slh_status slh_autotune(slh_ctx* ctx, int32_t lev, const slh_eom_params* p, int32_t reps, int32_t* chosen,
                        double* ms_out);

/* Autotuner of the diagnostics stage 1: as slh_autotune, timing reps
 * launches of stage 1 with the fused winding and energy partials (reads the
 * state, writes SLH_BUF_YA, SLH_BUF_D and the level's energy partials), and
 * keeps the fastest variant as the level's diagnostics tile
 * (slh_set_diag_tile).  Fills the level's ghost cells first (alpha = 1, as
 * slh_fill_ghosts), since the winding's cost depends on the values it reads.
 * Discards the partials of the last fused stage 1, so a
 * following slh_reduce_energy mode 1 fails with STATE until the next fused
 * step.  Synchronises.  Errors: INVALID_ARG, STATE, CUDA. */
slh_status slh_autotune_diag(slh_ctx* ctx, int32_t lev, const slh_eom_params* p, int32_t reps, int32_t* chosen,
                             double* ms_out);

/* Allocation-free energy reduction (the paper has no counterpart: this is a
 * service for embedders).  For callers that cannot call cudaMalloc -- code
 * running inside another library's stream-ordered section or a host callback
 * where allocating would synchronise or is forbidden, or an embedder whose
 * memory budget is handed out by its own allocator.  Computes the same five
 * numbers as slh_reduce_energy for one periodic box, here for a dense
 * lattice the caller owns: fields_dev holds psi1, psi2, Pi1, Pi2 as four
 * consecutive n^3 arrays (x fastest), FP64 (prec SLH_F64) or FP32
 * (SLH_F32_KAHAN); dx the spacing, eta the conformal time of the
 * coefficients, p the Laplacian order and potential; out_dev receives the
 * five doubles on the device, asynchronously on stream (a cudaStream_t).
 * Nothing is allocated: the per-plane partial sums live in one fixed
 * 128 KiB array in device global memory that is part of the library image
 * (every GPU that loads the library holds it until the process exits),
 * which limits the lattice side to n <= 4096 (larger n: SLH_ERR_OUT_OF_RANGE).
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  Every call overwrites the scratch rows it uses before
 * reading them, so nothing needs clearing, but calls that overlap on the GPU
 * (other streams, other threads) share the array and race.
 * Errors: INVALID_ARG, OUT_OF_RANGE, CUDA. */
slh_status slh_energy_noalloc(const void* fields_dev, int32_t n, int32_t prec, double dx, double eta,
                              const slh_eom_params* p, double* out_dev, void* stream);

/* Measured FMA issue rate of the current device (the ALU roofline of the
 * FP64 form, whose ~56 FP64 operations per cell and stage outweigh its
 * HBM traffic on a part that issues FP64 at a small fraction of its FP32
 * rate).  prec SLH_F64 (double FMAs) or SLH_F32_KAHAN (float FMAs).  A grid
 * of 8 CTAs of 256 threads per SM, each thread running 8 independent fma
 * recurrences, is timed with CUDA events on the legacy default stream, best
 * of reps (1..100) launches of ~15-80 ms each after one warm-up launch;
 * *fma_per_s receives fused multiply-adds per second for the whole device
 * (one FMA = 2 flops).  Synchronises the device; allocates nothing.
 * Errors: INVALID_ARG, CUDA. */
slh_status slh_alu_rate(int32_t prec, int32_t reps, double* fma_per_s);

/* Self-test of the bounded-wait path: launches one CTA that waits, for at
 * most `polls` polls (1..2^22), on an mbarrier phase that never completes
 * and latches the timeout exactly as the stage kernel's waits do.  The next
 * slh_sync returns SLH_ERR_TIMEOUT and clears it; the context stays usable.
 * Errors: INVALID_ARG, CUDA. */
slh_status slh_selftest_wait_timeout(slh_ctx* ctx, int64_t polls);

/* Wait for the stream and return any latched device error (then clear it). */
slh_status slh_sync(slh_ctx* ctx);

/* Profiling: when enabled, CUDA events bracket every launch and the device
 * time per kind (SLH_PROF_*) is accumulated; slh_profile_read synchronises
 * and returns the total milliseconds, the number of launches and the
 * algorithmic bytes those launches moved (field values read + written per
 * valid cell, ghost and halo re-reads excluded).  enable 0/1; reset clears.
 * While profiling is enabled slh_advance launches directly (no graph).
 * The host-phase kinds (SLH_PROF_REGRID_*, SLH_PROF_GRAPH_CAPTURE) give host
 * wall-clock milliseconds and the number of phases, always recorded. */
slh_status slh_profile(slh_ctx* ctx, int32_t enable, int32_t reset);
slh_status slh_profile_read(slh_ctx* ctx, int32_t kind, double* ms, int64_t* launches,
                            double* alg_bytes);

#ifdef __cplusplus
}
#endif
#endif /* SLH_H */
