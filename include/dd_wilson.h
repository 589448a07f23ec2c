/*
 * dd_wilson.h — C ABI of the GB300 (sm_103a) Wilson-clover library.
 *
 * The library applies the Wilson-clover Dirac operator of lattice QCD and
 * solves D x = b with FGMRES.  Operator and algorithms follow "Accelerating
 * Lattice QCD Simulations using GPUs" (T. Matthaei, 2023):
 *   D (Eq. 1.13 with a = 1)          (D psi)(x) = A(x) psi(x)
 *                                     - 1/2 sum_mu ((I - gamma_mu) (x) U_mu(x)) psi(x + mu)
 *                                     - 1/2 sum_mu ((I + gamma_mu) (x) U_mu^H(x - mu)) psi(x - mu)
 *   self coupling A(x) (Eq. 1.11, 1.12, 2.5)
 *                                     = (m0 + 4) I - (c_sw/32) sum_{mu,nu} gamma_mu gamma_nu (x) (Q_munu - Q_numu)
 *   FGMRES (Section 1.2, Algorithm 2).
 * Additions that the thesis does not have: the even-odd Schur operator,
 * FP32 / FP16-storage arithmetic with FP64 iterative refinement, multiple
 * right-hand sides, batched uneven lattices and the link derivative.
 *
 * Conventions
 *   dims = {nT, nZ, nY, nX}; every extent must be even and >= 2.
 *   site index (lexicographic, X fastest) = ((t*nZ + z)*nY + y)*nX + x.
 *   direction mu = 0..3 for T, Z, Y, X (Eq. 1.7, 1.8).
 *   spinor component = 3*spin + colour (Eq. 1.2).
 *   gamma matrices: Euclidean chiral basis,
 *     gamma_X,Y,Z = [[0, -i sigma_1,2,3], [i sigma_1,2,3, 0]], gamma_T = [[0, I], [I, 0]],
 *     gamma_5 = gamma_X gamma_Y gamma_Z gamma_T = diag(1, 1, -1, -1).
 *   time boundary: the fermion hop across t = nT-1 <-> 0 is multiplied by
 *     t_bc (-1 antiperiodic, +1 periodic); Z, Y, X are periodic.
 *   parity of a site = (t + z + y + x) mod 2 (0 even, 1 odd).
 *
 * Field layouts (argument `layout`)
 *   DD_LAYOUT_CANONICAL       device memory, complex double interleaved,
 *                             [nrhs][nsites][4 spin][3 colour].
 *   DD_LAYOUT_CANONICAL_HOST  the same shape in host memory (pinned memory is
 *                             faster); the call copies in and out itself and
 *                             returns after the result has reached the host.
 *   DD_LAYOUT_NATIVE          device memory in the library's native layout for
 *                             the precision (see dd_field_bytes).
 *   DD_LAYOUT_NATIVE_PAIRED   device memory in the paired-RHS layout (FP32 and
 *                             FP16 only, nrhs even; same bytes as native):
 *                             the same component of RHS 2j and 2j + 1 side by
 *                             side, for the packed paired stencil.
 *   For the full-lattice operators (DD_OP_D, DD_OP_DH) nsites = V.  For the
 *   even-odd operators (DD_OP_DHAT, DD_OP_DHAT_H) fields live on odd sites
 *   only: nsites = V/2, in increasing lexicographic order.
 *
 * Native layout (all device memory; Vh = V/2; N = nrhs; a "half field" holds
 * the sites of one parity, site k of parity p being the k-th site of that
 * parity in lexicographic order):
 *   FP64 half field: [12 components][Vh][N] of complex double (16 B).
 *   FP32 half field: [6 component pairs][Vh][N] of float4 (re, im of
 *                    components 2c and 2c + 1).
 *   FP16 half field: [3 component quads][Vh][N] of 8 halves (re, im of
 *                    components 4c .. 4c + 3, divided by the site scale),
 *                    then [Vh][N] float scales (max |re|, |im| over the 24 reals).
 *   A full field is the even half field followed by the odd half field.
 * Paired-RHS layout (nrhs = N even, NP = N / 2; pair j holds RHS 2j and 2j + 1):
 *   FP32 half field: [12 components][Vh][NP] of float4
 *                    (re RHS 2j, re RHS 2j + 1, im RHS 2j, im RHS 2j + 1).
 *   FP16 half field: [6 component pairs][Vh][NP] of 4 half2 (re and im of
 *                    component 2c, then of 2c + 1; each half2 holds RHS 2j and
 *                    2j + 1, divided by their own site scales), then [Vh][N]
 *                    float scales as in the native FP16 layout.
 *   Full fields as for the native layout.  Canonical applies of D, D^H, Dhat
 *   and Dhat^H with an even nrhs in FP32 or FP16 run on this layout
 *   internally; the result is bit-identical to the native-layout apply.
 *
 * Ownership: handles own the device memory they allocate.  Field pointers
 * passed to calls belong to the caller and are never freed or retained.
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls on device layouts only enqueue work and return; calls on
 * DD_LAYOUT_CANONICAL_HOST and dd_solve synchronise the stream.
 * Errors: every call returns a status (DD_OK = 0, negative on error); it never
 * aborts.  dd_last_error_detail() describes the last error of the calling
 * thread.
 *
 * Environment (each read once per process, at first use; all optional):
 *   DD_RECON=r          form of the compressed FP32 / FP16 link copies made
 *                       at dd_gauge_create for SU(3) links (see
 *                       dd_gauge_compress_links): 12 two rows (default), 8
 *                       eight reals for FP32 (two rows where they do not
 *                       rebuild to 1e-6) and two rows for FP16, 0 none (the
 *                       single-RHS kernels then read three rows).
 *   DD_RHS_BLOCK=n      largest RHS block of the multi-RHS stencil (1, 2 or
 *                       4; default 4; 1 gives one thread per site and RHS,
 *                       also for canonical applies, which otherwise take the
 *                       paired-RHS stencil for an even nrhs).
 *   DD_ZBLOCK=d         Z-slab depth of the traversal (a divisor of nZ; 0 =
 *                       nZ); default: the deepest slab within 30 MB.
 *   DD_HOST_CHUNKS=c    time-slice chunks of the pipelined host-buffer
 *                       apply (default 48, at most nT).
 *   DD_FUSED_NORM=0     the CG preconditioner of dd_solve takes its norms
 *                       from separate reductions instead of the stencil
 *                       launch (read at each dd_solve).
 *   DD_STAGE=1          opt-in row-staged stencil for full-lattice FP32
 *                       applies (canonical applies then keep the native
 *                       layout; slower; DD_STAGE_SLOTS sets its ring depth,
 *                       DD_STAGE_NARROW=1 allows its narrow-row variant,
 *                       DD_STAGE_WAIT_TEST=1 makes one of its waits expire
 *                       so that tests can check dd_device_status).
 */
#ifndef DD_WILSON_H
#define DD_WILSON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define DD_OK 0
#define DD_ERR_ARG (-1)            /* bad argument (null pointer, size, enum) */
#define DD_ERR_OOM (-2)            /* device or host allocation failed */
#define DD_ERR_CUDA (-3)           /* a CUDA call failed */
#define DD_ERR_SINGULAR (-4)       /* a self-coupling block could not be inverted */
#define DD_ERR_NOT_CONVERGED (-5)  /* solver hit its iteration limit; x holds the best iterate */
#define DD_ERR_TIMEOUT (-6)        /* a bounded device wait gave up */
#define DD_ERR_UNSUPPORTED (-7)    /* combination not built (e.g. precision not created) */

/* ---- precisions (bit flags for masks) ---- */
#define DD_PREC_F64 1  /* FP64 storage and arithmetic */
#define DD_PREC_F32 2  /* FP32 storage and arithmetic */
#define DD_PREC_F16 4  /* FP16 storage (spinors with a per-site FP32 scale), FP32 arithmetic */
/* FP64-accurate arithmetic in pairs of FP32 numbers x = h + l, |l| <= ulp(h)/2
 * (Dekker's double-word arithmetic: about 48 significant bits, from the FP32
 * pipes), with links, blocks and native fields stored as such pairs: one
 * complex = (re.h, re.l, im.h, im.l), 16 bytes, in the FP64 layouts (native
 * fields of this precision have the FP64 byte count).  Accepted by
 * dd_gauge_create / dd_gauge_generate / dd_clover_create (precision masks),
 * dd_field_bytes, dd_pack, dd_unpack and dd_apply (all operators, native
 * and canonical layouts except the paired one), and as dd_solve's
 * inner_prec (FP64 Krylov vectors, split into pairs as the stencil loads
 * them, 2^-46 relative; preconditioners none, normal and CGNR); not by SAP,
 * AMG, the batch, the domain decomposition or dd_force (DD_ERR_ARG or
 * DD_ERR_UNSUPPORTED).  Canonical inputs are split into pairs exactly to
 * about 2^-48 relative; results are rounded to FP64 by h + l. */
#define DD_PREC_DF64 8

/* ---- operators ---- */
#define DD_OP_D 0       /* D, Eq. 1.13 */
#define DD_OP_DH 1      /* D^H = gamma5 D gamma5 */
#define DD_OP_DHAT 2    /* Dhat = A_oo - D_oe A_ee^{-1} D_eo on odd sites */
#define DD_OP_DHAT_H 3  /* Dhat^H = gamma5 Dhat gamma5 */
#define DD_OP_SC 4      /* D_sc alone (Eq. 2.5): the self coupling A(x) psi(x) */

/* ---- layouts ---- */
#define DD_LAYOUT_CANONICAL 0
#define DD_LAYOUT_CANONICAL_HOST 1
#define DD_LAYOUT_NATIVE 2
#define DD_LAYOUT_NATIVE_PAIRED 3
/* complex64 canonical fields [N][V or V/2][4][3] (float re, im), on the
 * device or on the host: dd_apply only (native layout inside; FP32 / FP16
 * applies read and write them without the complex128 round trip, so the
 * host-buffer apply moves half the bytes; FP64 / FP32-pair applies take
 * their inputs at FP32 precision). */
#define DD_LAYOUT_CANONICAL_C64 4
#define DD_LAYOUT_CANONICAL_HOST_C64 5

typedef struct dd_lattice dd_lattice;
typedef struct dd_gauge dd_gauge;
typedef struct dd_clover dd_clover;
typedef struct dd_batch dd_batch;
typedef struct dd_amg dd_amg;

/* Human-readable name of a status code (static string). */
const char* dd_error_string(int status);
/* Detail of the calling thread's last error (static per thread, never NULL). */
const char* dd_last_error_detail(void);
/* Library version, major * 10000 + minor * 100 + patch. */
int dd_version(void);

/*
 * Lattice of dims[4] = {nT, nZ, nY, nX} (Eq. 1.9), all even and >= 2, with
 * V = nT nZ nY nX < 2^31.  t_bc = -1 (antiperiodic in time) or +1.
 * Host-only object; DD_ERR_ARG on bad sizes.
 */
int dd_lattice_create(const int dims[4], int t_bc, dd_lattice** out);
int dd_lattice_destroy(dd_lattice* lat);
int64_t dd_lattice_volume(const dd_lattice* lat);

/* Rows per link that single-RHS applies read in precision `prec`
 * (DD_PREC_F64 / F32 / F16): 3, or 2 for DD_PREC_F32 and DD_PREC_F16 when
 * every link passed to dd_gauge_create is an SU(3) matrix to 1e-6 (max of
 * |U U^H - 1| and |det U - 1|).  The gauge handle then holds second FP32 and
 * FP16 copies with rows 0 and 1 only (FP32 192 instead of 288 bytes per site,
 * FP16 96 instead of 144), and single-RHS stencils rebuild row 2 as the
 * complex conjugate of the cross product of rows 0 and 1, which holds for
 * SU(3) matrices (Section 1.1 of the thesis defines the links as SU(3)
 * elements); several-RHS launches keep reading three rows.  The environment
 * variable DD_RECON=0, read at gauge creation, skips the two-row copies.
 * DD_ERR_UNSUPPORTED if the copy of `prec` was not created.  With the
 * eight-real FP32 copy (dd_gauge_compress_links) this returns 3 for
 * DD_PREC_F32: use dd_gauge_link_reals. */
int dd_gauge_stored_rows(const dd_gauge* g, int prec);

/* Real numbers per link that single-RHS applies read in precision `prec`:
 * 18 (three rows), 12 (two rows, DD_PREC_F32 / F16) or 8 (DD_PREC_F32).
 * DD_ERR_ARG / DD_ERR_UNSUPPORTED as dd_gauge_stored_rows. */
int dd_gauge_link_reals(const dd_gauge* g, int prec);

/* Choose the compressed link copy that single-RHS applies of precision
 * `prec` (DD_PREC_F32 or DD_PREC_F16) read (Section 2.3 stores the links of
 * the stencil; an SU(3) matrix has 8 real degrees of freedom, Section 1.1):
 *   reals = 18  no copy: the three-row links (FP32 288 bytes per site, FP16
 *               144);
 *   reals = 12  rows 0 and 1 (FP32 192 bytes per site, FP16 96), row 2
 *               rebuilt as the complex conjugate of the cross product of rows
 *               0 and 1 (FP16: exact products of the stored values, FP32
 *               sums, one rounding to FP16);
 *   reals = 8   FP32 only: two float4 words per link (128 bytes per site):
 *               W = S U C, C a cyclic column shift putting the largest
 *               element of row 0 first, S keeping rows 1, 2 or replacing them
 *               by (row 2, -row 1) so that the stored lower entry of column 0
 *               is the smaller one; stored are W01, W02, W10 and the phases
 *               of W00 and W20 (divided by pi), the shift and swap in the
 *               lowest mantissa bits of three of the stored values.  The
 *               stencil rebuilds |W00| and |W20| from the unit norms of row 0
 *               and column 0, W11 and W12 from the orthogonality of rows 0
 *               and 1 and from W20 = conj(W01 W12 - W02 W11) (a 2x2 solve of
 *               determinant |W01|^2 + |W02|^2), and row 2 as for 12.
 * 12 and 8 need links of `prec` in the handle and every link SU(3) to 1e-6
 * (dd_gauge_stored_rows); 8 also checks every rebuilt element against the
 * FP64 link and keeps the previous form when one is off by more than 1e-6
 * (the parametrisation is singular where W01 = W02 = 0, e.g. unit links).
 * Several-RHS launches always read the three-row links.  Domains made by
 * dd_decomp_create copy the FP32 two-row form current at their creation
 * (they read three rows with the eight-real form and in FP16).
 * Synchronises the device; no launch may use the handle meanwhile.
 * DD_ERR_ARG for another `prec` or `reals`; DD_ERR_UNSUPPORTED (previous form
 * kept) when the links or the precision do not allow the form. */
int dd_gauge_compress_links(dd_gauge* g, int prec, int reals);

/*
 * Gauge field U_mu(x) in SU(3) (Section 1.1), given as complex double
 * [V][4 mu][3][3] (row-major colour matrices; U_mu(x) links x to x + mu).
 * `location` 0 = host pointer, 1 = device pointer.  The library copies the
 * links into its native layout in every precision of `prec_mask` (FP64 is
 * always kept).  The caller keeps ownership of U.  The lattice must outlive
 * the gauge handle.
 */
int dd_gauge_create(const dd_lattice* lat, const double* U, int location, unsigned prec_mask, dd_gauge** out);
/*
 * Synthetic gauge field generated on the device (the thesis' gauge
 * configurations are not public; this generator stands in for them and is not
 * part of the thesis).  Link U_mu(x) = exp(i eps H) with H = (A + A^H)/2 -
 * (tr A_re / 3) I traceless Hermitian, A a 3x3 matrix of complex Gaussians
 * (Re, Im i.i.d. N(0, 1)); U is special unitary, the SU(3) element of
 * Section 1.1.  The Gaussians come from a counter-based stream, so every link
 * is drawn independently of launch shape and thread count:
 *   key = mix64(seed), word k = mix64(key + (k + 1) * 0x9E3779B97F4A7C15)
 *   (SplitMix64, Steele, Lea and Flood 2014); Gaussian pair number
 *   n = (4 x + mu) * 9 + (3 a + b) for entry (a, b) of A at link (x, mu), from
 *   u1 = ((word(2n) >> 11) + 1) 2^-53, u2 = (word(2n + 1) >> 11) 2^-53 by
 *   Box-Muller: sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).
 * The exponential is a 14-term Taylor series with scaling and squaring.
 * Layouts and precision copies as for dd_gauge_create (FP64 always kept);
 * the result equals dd_gauge_create of the same field generated on the host
 * to rounding (about 1e-15).  eps must be finite and >= 0 (DD_ERR_ARG
 * otherwise); the benchmark configurations use eps = 0.3, seed 20240700.
 * Synchronises the device.  The lattice must outlive the gauge handle.
 */
int dd_gauge_generate(const dd_lattice* lat, uint64_t seed, double eps, unsigned prec_mask, dd_gauge** out);
int dd_gauge_destroy(dd_gauge* g);
/* Copy the FP64 links back out as complex double [V][4][3][3] to host (location 0) or device (1). */
int dd_gauge_download(const dd_gauge* g, double* U, int location);

/*
 * Operator handle: builds the self coupling A(x) of Eq. 2.5 from the links on
 * the device (Q_munu per Eq. 1.12, clover term per Eq. 1.11, mass term m0 + 4)
 * as two Hermitian 6x6 blocks per site (upper and lower chirality; the
 * clover term commutes with gamma5 in the chiral basis), and A_ee^{-1} on even
 * sites in FP64.  Lower-precision copies are made for `prec_mask`.
 * DD_ERR_SINGULAR if an even-site block has no inverse.  The gauge handle must
 * outlive the operator.
 */
int dd_clover_create(const dd_gauge* g, double m0, double csw, unsigned prec_mask, dd_clover** out);
int dd_clover_destroy(dd_clover* op);
/* Self coupling of every site as dense 12x12 complex double [V][12][12] in
 * host memory (for checking). */
int dd_clover_download(const dd_clover* op, double* A_host);

/*
 * Bytes of one native field: subset 0 = full lattice, 1 = one parity (V/2
 * sites), for `nrhs` right-hand sides in precision `prec`.
 */
size_t dd_field_bytes(const dd_clover* op, int prec, int subset, int nrhs);

/*
 * Convert between the canonical layout (device, complex double) and the
 * native layout of precision `prec`.  subset 0: full field ([nrhs][V][12]
 * canonical); 1: odd sites ([nrhs][V/2][12]); 2: even sites.
 * Enqueued on `stream`.
 */
int dd_pack(const dd_clover* op, int prec, int subset, const double* canon, void* native, int nrhs, void* stream);
int dd_unpack(const dd_clover* op, int prec, int subset, const void* native, double* canon, int nrhs, void* stream);
/* The same for the paired-RHS layout (prec DD_PREC_F32 or DD_PREC_F16, nrhs
 * even and >= 2; DD_ERR_ARG otherwise).  The layout itself is not in the
 * thesis: it serves the packed FP32x2 stencil of dd_apply. */
int dd_pack_paired(const dd_clover* op, int prec, int subset, const double* canon, void* paired, int nrhs,
                   void* stream);
int dd_unpack_paired(const dd_clover* op, int prec, int subset, const void* paired, double* canon, int nrhs,
                     void* stream);

/*
 * out = OP in for `nrhs` right-hand sides at precision `prec` (the precision
 * must have been created in both the gauge and the operator handle).
 * op: DD_OP_D, DD_OP_DH, DD_OP_SC (full lattice) or DD_OP_DHAT, DD_OP_DHAT_H
 * (odd sites).  in and out must not overlap.  Canonical layouts are converted
 * to and from the native layout inside the call, using workspace owned by the
 * operator handle (allocated on first use and kept).
 * DD_LAYOUT_NATIVE_PAIRED (DD_OP_D, DD_OP_DH, DD_OP_DHAT, DD_OP_DHAT_H with
 * prec DD_PREC_F32 or DD_PREC_F16 and an even nrhs) runs the packed paired
 * stencil: one thread per output site and pair of right-hand sides.  FP32:
 * each arithmetic step the FP32 operation of the native-layout kernel
 * (results are bit-identical).  FP16: spin projection and colour products in
 * half2 arithmetic on the stored values (FP16 sums; results within about
 * 1e-3 relative of the native-layout kernel, which widens to FP32 first), the
 * hop sums and the self coupling in FP32.  Canonical layouts with an even
 * nrhs take this stencil too.  DD_ERR_ARG for an odd nrhs or another
 * precision, DD_ERR_UNSUPPORTED for DD_OP_SC.
 * Enqueued on `stream`; DD_LAYOUT_CANONICAL_HOST synchronises it.
 */
int dd_apply(dd_clover* op, int which, int prec, const void* in, void* out, int nrhs, int layout, void* stream);

/* ---- solver (Algorithm 2 inside FP64 iterative refinement) ---- */
typedef struct {
  double tol;          /* stop when ||b - D x|| < tol ||b|| (full-system FP64 residual), e.g. 1e-10 */
  int restart;         /* Krylov dimension m of FGMRES(m), e.g. 30 */
  int max_restarts;    /* restart cycles allowed per inner solve */
  int max_outer;       /* refinement steps allowed (1 with inner_prec = F64 means a plain FP64 solve) */
  int inner_prec;      /* DD_PREC_F64, DD_PREC_F32, DD_PREC_F16 (FP16 links/clover, FP32 vectors) or
                          DD_PREC_DF64 (FP32-pair arithmetic, FP64 vectors) */
  double inner_tol;    /* relative residual reduction asked of each inner solve, e.g. 1e-6 */
  int even_odd;        /* 1: inner solves use Dhat on odd sites; 0: D on the full lattice */
  int verbose;         /* 1: print progress lines to stderr */
  int precond;         /* preconditioner M_j of Algorithm 2: DD_PRECOND_NONE (M = I),
                          DD_PRECOND_NORMAL (M^{-1} = A^H, so A M^{-1} = A A^H is Hermitian
                          positive definite and restarted FGMRES cannot stagnate),
                          DD_PRECOND_CGNR (flexible: CG steps on the normal equations),
                          DD_PRECOND_SAP (flexible: Schwarz cycles, see dd_sap),
                          DD_PRECOND_AMG (flexible: the two-level preconditioner `amg`) or
                          DD_PRECOND_CGNR16 (DD_PRECOND_CGNR with FP16 CG vectors) */
  int gs_passes;       /* classical Gram-Schmidt passes per Arnoldi step: 1, or 2 (re-orthogonalised) */
  int rhs_batch;       /* even-odd solves: right-hand sides solved together (0 = all); smaller
                          batches need proportionally less device memory */
  int precond_iters;   /* DD_PRECOND_CGNR / CGNR16: conjugate-gradient steps per preconditioner
                          application */
  int sap_block[4];    /* DD_PRECOND_SAP: block extents (T, Z, Y, X), as for dd_sap */
  int sap_cycles;      /* DD_PRECOND_SAP: red-black cycles per preconditioner application */
  int sap_mr_steps;    /* DD_PRECOND_SAP: minimal-residual steps per block solve */
  dd_amg* amg;         /* DD_PRECOND_AMG: the two-level preconditioner (dd_amg_create); its fine
                          precision must be that of the inner vectors (F64 for inner_prec F64,
                          F32 otherwise) and it must belong to the same operator */
  int refine_prec;     /* arithmetic of the refinement's operator applications on the FP64
                          iterate (r = b - D x, the even-odd preparation and reconstruction):
                          DD_PREC_F64 (default) or DD_PREC_DF64 (the FP32-pair stencil on the
                          same FP64 vectors, about 1e-14 relative, needs the DF64 copies in the
                          gauge and operator handles; DD_ERR_UNSUPPORTED without them).  The
                          reported true_residual is computed the same way. */
} dd_solve_params;

#define DD_PRECOND_NONE 0
#define DD_PRECOND_NORMAL 1
#define DD_PRECOND_CGNR 2  /* flexible M_j: precond_iters CG steps on A^H A z = A^H v_j */
#define DD_PRECOND_SAP 3   /* flexible M_j: sap_cycles Schwarz cycles on D (even-odd: the odd half of
                              the cycles applied to (0, v_j), D^{-1}'s odd-odd block being Dhat^{-1}) */
#define DD_PRECOND_AMG 4   /* flexible M_j: the two-level AMG preconditioner `amg` (even-odd: the odd
                              half of M^{-1} (0, v_j)) */
#define DD_PRECOND_CGNR16 5 /* DD_PRECOND_CGNR with the CG vectors r, p, A p and A^H r stored in FP16
                              (per-site scales; the iterate z_j in FP32): inner_prec DD_PREC_F16 (FP16
                              links and self coupling) or DD_PREC_F32 (FP32 ones) */

typedef struct {
  int converged;             /* 1 if every right-hand side met tol */
  int outer_iterations;      /* refinement steps */
  int inner_iterations;      /* Arnoldi steps summed over inner solves (max over RHS) */
  int restarts;              /* restart cycles summed over inner solves */
  int applies_inner;         /* operator applications inside inner solves */
  int applies_fp64;          /* FP64 operator applications (true residuals) */
  double true_residual;      /* max over RHS of ||b - D x|| / ||b|| in FP64 */
  double seconds;            /* wall time of the call */
} dd_stats;

/* Fill `p` with defaults: tol 1e-10, restart 30, max_restarts 100,
 * max_outer 30, inner_prec F32, inner_tol 1e-6, even_odd 1, precond NONE, gs_passes 1,
 * rhs_batch 0, precond_iters 32, sap_block {4, 4, 4, 4}, sap_cycles 1, sap_mr_steps 4, amg NULL. */
void dd_solve_params_default(dd_solve_params* p);

/*
 * Solve D x = b for `nrhs` right-hand sides.  b and x use `layout`
 * (canonical device or host; full lattice); x holds the initial guess on
 * entry and the solution on exit.  Convergence is judged on the FP64 true
 * residual of the full system.  Returns DD_ERR_NOT_CONVERGED (with x = best
 * iterate and stats filled) when limits are hit.  Synchronises `stream`.
 * `stats` may be NULL.
 * even_odd = 1: FP64 refinement runs on the odd-site system Dhat x_o = bhat_o
 * (x_o enters from the odd sites of x), x_e = A_ee^{-1} (b_e - D_eo x_o) is
 * formed at the end and the full residual verified; with host layout only one
 * batch of b / x is staged on the device at a time.
 * even_odd = 0: refinement and inner solves on the full lattice.
 */
int dd_solve(dd_clover* op, const dd_solve_params* params, const void* b, void* x, int nrhs, int layout,
             void* stream, dd_stats* stats);

/* ---- Schwarz alternating procedure (SAP) ----
 * z = M^{-1} v for the block smoother that the thesis names for DDalphaAMG
 * (Section 1.3), read as red-black multiplicative Schwarz with
 * non-overlapping blocks:
 *   the lattice is cut into blocks of block[0..3] = (b_T, b_Z, b_Y, b_X)
 *   sites aligned with the origin; every extent must hold an even number of
 *   blocks and a block at most 256 sites (DD_ERR_ARG otherwise); the colour
 *   of a block is the parity of the sum of its block coordinates;
 *   D_B is D restricted to block B with the hops that leave it dropped;
 *   from z = 0, r = v, each of `cycles` cycles treats the blocks of colour 0
 *   and then of colour 1: e_B = `mr_steps` minimal-residual steps on
 *   D_B e = r_B from e = 0 (q = D_B rho, alpha = q^H rho / q^H q,
 *   e += alpha rho, rho -= alpha q) on every block of the colour,
 *   z += e, r = v - D z.
 * v, z: full fields of `nrhs` right-hand sides in `layout` (canonical device
 * or host, or native); prec DD_PREC_F64 or DD_PREC_F32 (arithmetic and
 * native vectors), or DD_PREC_F16 (FP16 links and blocks, FP32 vectors;
 * canonical layouts only).  Workspace is owned by the operator handle.
 * Enqueued on `stream` (host layout synchronises).
 */
int dd_sap(dd_clover* op, int prec, const int block[4], int cycles, int mr_steps, const void* v, void* z, int nrhs,
           int layout, void* stream);

/* ---- two-level algebraic multigrid (AMG) preconditioner ----
 * Section 1.3: a coarse operator D_c that acts on the near kernel of D (the
 * eigenvectors of small |eigenvalue|) like D and couples nearest neighbours
 * only, a restriction R and prolongation P between the lattices built from
 * test vectors found in a setup phase, and the subspace correction
 * z <- z + P D_c^{-1} R r together with the SAP smoother as M_j of FGMRES
 * (Table 5.2: depth-one coarse lattices of 4^4 or 8^4 sites per coarse site,
 * 24 test vectors, 4 setup iterations).  The thesis gives no formulas for
 * P, R or the setup; the reading implemented here:
 *   aggregates: blocks of aggregate[0..3] sites aligned with the origin (each
 *   extent must divide the lattice extent), numbered lexicographically on the
 *   coarse lattice (X fastest), each with 2 n_tv coarse degrees of freedom,
 *   n_tv per chirality (spins 0, 1 and 2, 3);
 *   P: the n_tv test vectors restricted to (aggregate, chirality),
 *   orthonormalised by modified Gram-Schmidt in order; R = P^H;
 *   D_c = R D P (Galerkin);
 *   M^{-1} v = z with z = P D_c^{-1} R v (the coarse system solved by GMRES
 *   to coarse_tol), then z += SAP(v - D z) (sap_cycles cycles, 0 = none);
 *   setup: from the n_tv given vectors w0, init_sap_iters rounds of
 *   w_i <- SAP(w_i), then setup_iters rounds of w_i <- M^{-1} w_i with M
 *   built from the current w (every w_i normalised after each round);
 *   P and D_c are built from the final w.
 * Coarse vectors and D_c are FP64 on the device; D_c is stored per aggregate
 * A as nine 2 n_tv x 2 n_tv blocks, column-major: block 0 couples A with
 * itself, block 1 + 2 mu with the aggregate at +mu, 2 + 2 mu with -mu
 * (periodic on the coarse lattice).
 */
typedef struct {
  int aggregate[4];         /* aggregate extents (T, Z, Y, X) */
  int n_tv;                 /* test vectors: 4, 8 or 16 */
  int setup_iters;          /* rounds of w_i <- M^{-1} w_i */
  int init_sap_iters;       /* initial rounds of w_i <- SAP(w_i) */
  int sap_block[4];         /* SAP block extents (as for dd_sap) */
  int sap_cycles;           /* post-smoothing cycles per application (0: no smoothing) */
  int sap_mr_steps;         /* MR steps per SAP block solve */
  double coarse_tol;        /* relative residual asked of the coarse GMRES */
  int coarse_restart;       /* its restart length (1 .. 32) */
  int coarse_max_restarts;  /* its restart cycles at most */
} dd_amg_params;

/* Defaults: aggregate {4,4,4,4}, n_tv 8, setup_iters 2, init_sap_iters 2,
 * sap_block {4,4,4,4}, sap_cycles 1, sap_mr_steps 4, coarse_tol 5e-2,
 * coarse_restart 16, coarse_max_restarts 4. */
void dd_amg_params_default(dd_amg_params* p);
/* Run the setup and return the preconditioner.  prec: DD_PREC_F64 (FP64
 * everywhere), DD_PREC_F32, or DD_PREC_F16 (FP16 links and blocks, FP32
 * vectors) for P, the build of D_c and the smoothing.  w0: the initial test
 * vectors, canonical device fields [n_tv][V][12] complex double (the caller
 * draws them; they are not kept).  DD_ERR_ARG on bad parameters,
 * DD_ERR_SINGULAR if the vectors are linearly dependent on an aggregate.
 * Synchronises the device.  `op` must outlive the handle. */
int dd_amg_create(dd_clover* op, int prec, const dd_amg_params* params, const double* w0, dd_amg** out);
int dd_amg_destroy(dd_amg* amg);
/* Coarse lattice extents, coarse degrees of freedom per aggregate (2 n_tv),
 * setup wall time, and Arnoldi steps of the last coarse solve (each pointer
 * may be NULL). */
int dd_amg_info(const dd_amg* amg, int* coarse_dims4, int* dof_per_aggregate, double* setup_seconds,
                int* last_coarse_steps);
/* D_c to host memory: complex double [n_agg][9][2 n_tv][2 n_tv] as stored
 * (column-major blocks).  Synchronises the device. */
int dd_amg_coarse_download(const dd_amg* amg, double* Dc_host);
/* z = M^{-1} v for nrhs full fields: canonical device fields (complex
 * double) or native fields of the handle's fine precision.  Workspace is
 * owned by the handle (and the operator handle's canonical buffers); calls on
 * one handle must not overlap. */
int dd_amg_apply(dd_amg* amg, const void* v, void* z, int nrhs, int layout, void* stream);

/* ---- link derivative (not in the thesis) ----
 * For L = Re <phi, D psi> = Re sum_x phi(x)^H (D psi)(x), writes per link
 *   G_mu(x) = dL/dRe U_mu(x) + i dL/dIm U_mu(x)           (if G != NULL)
 *   F_mu(x) = P(G_mu(x) U_mu(x)^H), P(M) = (M - M^H)/2 - tr(M - M^H)/6 I
 *                                                          (if F != NULL)
 * as complex double [V][4][3][3] on the device.  phi, psi: canonical device
 * fields [nrhs][V][12]; contributions of all right-hand sides are summed.
 * with_clover = 0 holds the self coupling fixed (hopping terms only); 1 also
 * differentiates A(x) through Q_munu (Eq. 1.11, 1.12).  prec: DD_PREC_F64 or
 * DD_PREC_F32 (arithmetic precision; outputs are FP64).  Enqueued on stream.
 * DD_PREC_F32 accumulates in a workspace owned by the operator handle
 * (80 bytes per link, kept between calls), so FP32 force calls on one handle
 * must not overlap on the GPU.
 */
int dd_force(dd_clover* op, int prec, const double* phi, const double* psi, int nrhs, int with_clover, double* G,
             double* F, void* stream);

/* ---- batched uneven lattices ----
 * A batch groups operator handles of different lattices (FP32 or FP16
 * precision) and applies D to all of them in one persistent kernel launch.
 * Work items are (lattice, site tile, RHS block) triples; the tile and RHS
 * block shapes come from the autotuner (dd_batch_tune) or defaults.
 */
int dd_batch_create(dd_clover* const* ops, int count, int prec, const int* nrhs, dd_batch** out);
int dd_batch_destroy(dd_batch* b);
/* ins[i], outs[i]: native device fields of operator i (full lattice, nrhs[i] RHS). */
int dd_apply_batched(dd_batch* b, const void* const* ins, void* const* outs, void* stream);
/* Field layout of the batch: DD_LAYOUT_NATIVE (default) or
 * DD_LAYOUT_NATIVE_PAIRED, under which the lattices with an even RHS count
 * take paired-RHS fields (dd_pack_paired; their launches run the packed
 * FP32x2 stencil) and the others native fields.  The paired layout runs one
 * launch per lattice on forked streams (the persistent shapes take native
 * fields only) and drops a captured graph.  DD_ERR_ARG for another layout. */
int dd_batch_set_layout(dd_batch* b, int layout);
/* Time candidate launch shapes on `stream` and keep the fastest; optional
 * report of the chosen shape (slots per tile, threads per block, CTAs per SM,
 * where 0 CTAs per SM means one CTA per work item instead of a persistent
 * grid, and -1 one launch per lattice with its own best single-lattice kernel
 * on parallel streams, which dd_apply_batched_graph captures as parallel
 * graph branches). */
int dd_batch_tune(dd_batch* b, const void* const* ins, void* const* outs, void* stream, int* chosen3);
/* Capture the batched launch in a CUDA graph on first call and replay it
 * afterwards (same pointers required; DD_ERR_ARG otherwise). */
int dd_apply_batched_graph(dd_batch* b, const void* const* ins, void* const* outs, void* stream);

/* ---- domain decomposition (Sections 2.1, 2.2, Algorithm 3) ----
 * The lattice of an operator handle split into grid[0] x grid[1] x grid[2] x
 * grid[3] hyper-rectangular local lattices P_i, one per virtual rank on this
 * GPU; rank i has lexicographic grid coordinates (T, Z, Y, X; X fastest) and
 * local site (t, z, y, x) is global site (t + off_T, ..., x + off_X) with
 * off = coordinate * local extent.  Every global extent must divide into
 * grid[mu] even local extents.  Each rank holds its own copy of the links,
 * the self-coupling blocks and A_ee^{-1} of every precision of `op`, native
 * input, output and work fields (the full-field native layout of its local
 * lattice) and face buffers.  An apply evaluates the neighbour coupling as
 * Algorithm 3 does, for every split direction mu: each rank projects the spin
 * components of its lowest mu slice, (I -/+ gamma_mu) psi (lambda), and of its
 * highest slice times U_mu(x)^H (chi), 6 complex per site and RHS, sends
 * lambda to the rank at -mu and chi to the rank at +mu (device-to-device
 * copies into the receiver's own buffer, on a stream of the handle), computes
 * its interior sites meanwhile, and finishes the sites next to a seam once
 * the messages have arrived.  Directions with grid[mu] = 1 wrap inside the
 * rank.  The results equal the single-domain dd_apply bit for bit where that
 * runs the one-thread-per-(site, RHS) stencil (one RHS, an odd RHS count, or
 * FP64), and to rounding otherwise.  `op` must outlive the handle.
 */
typedef struct dd_decomp dd_decomp;
int dd_decomp_create(const dd_clover* op, const int grid[4], dd_decomp** out);
int dd_decomp_destroy(dd_decomp* d);
/* Number of ranks (> 0), or a negative status; fills the rank's grid
 * coordinates, global offset, local extents and number of sites next to a
 * split seam (each pointer may be NULL). */
int dd_decomp_info(const dd_decomp* d, int rank, int* coord4, int* offset4, int* local4, int64_t* boundary_sites);
/* Copy a global native field of precision `prec` (subset 0: full lattice;
 * 1: odd sites, the Dhat layout) into every rank's input field (scatter), or
 * every rank's output field back into a global native field (gather, with the
 * precision and RHS count of the last scatter).  Enqueued on `stream`. */
int dd_decomp_scatter(dd_decomp* d, int prec, int subset, const void* global_native, int nrhs, void* stream);
int dd_decomp_gather(dd_decomp* d, int prec, int subset, void* global_native, int nrhs, void* stream);
/* output = OP input on every rank: DD_OP_D, DD_OP_DH (full fields) or
 * DD_OP_DHAT, DD_OP_DHAT_H (odd halves; two exchange rounds, one per stencil
 * launch).  Precision and RHS count of the last scatter.  Enqueued on
 * `stream`. */
int dd_decomp_apply(dd_decomp* d, int which, int prec, int nrhs, void* stream);
/* dots[r] = sum over all ranks of sum_x output_r(x)^H input_r(x) (subset 0
 * full fields, 1 odd halves): each rank's partial sum over its own sites, then
 * the sum over ranks in rank order (the allreduce of the Gram-Schmidt inner
 * products in a decomposed Algorithm 2).  FP64 or FP32 fields; written to
 * host memory [nrhs][2] after synchronising `stream`. */
int dd_decomp_dot(dd_decomp* d, int prec, int subset, int nrhs, double* dots_host, void* stream);

/* ---- vector operations on canonical device fields (FP64) ----
 * dots[r] = <a_r, b_r> = sum a_r^H b_r over `nsites` sites, for r < nrhs;
 * written to host memory after synchronising the stream. */
int dd_dot(const double* a, const double* b, int64_t nsites, int nrhs, double* dots_host /*[nrhs][2]*/, void* stream);

/* Allocation-free variant of dd_dot.  The thesis has no counterpart; it is
 * for callers that cannot allocate device memory when they need the inner
 * products: code whose memory pool already owns the free device memory,
 * callers under a hard allocation cap, and phases where cudaMalloc or cudaFree
 * would synchronise the device.  Same arguments and result as dd_dot; no
 * cudaMalloc, cudaFree or allocating library routine is called.
 * Scratch: a fixed device array of about 20 KB inside the library, held on
 * every GPU that loads the library until the process exits.  Its device
 * address is looked up on the first call made on each device, so make that
 * first call before any stream capture.  All calls share the array and it
 * keeps the last call's contents (nothing in it has to start at zero), so
 * calls that overlap on the GPU (other streams or threads) race.
 * Limit: nrhs <= 64, else DD_ERR_ARG.  Synchronises `stream`. */
int dd_dot_noalloc(const double* a, const double* b, int64_t nsites, int nrhs, double* dots_host /*[nrhs][2]*/,
                   void* stream);

/* ---- arithmetic peak probe ----
 * The method of Section 3.1 / Table 3.1 of the thesis: many threads each run
 * long register-only chains of floating-point operations (here eight
 * independent fused multiply-add chains).  Writes the measured rate in FLOP/s
 * (an FMA counts as 2) for DD_PREC_F64 or DD_PREC_F32 on the current device.
 * Synchronises `stream`. */
int dd_probe_flops(int prec, double* flops_per_second, void* stream);

/* ---- device wait status ----
 * Kernels that wait on asynchronous copies (the row-staged stencil of
 * dd_apply, which moves neighbour rows into shared memory with bulk copies
 * completing on mbarriers) bound every wait in time; a wait that expires
 * makes the kernel record it in a device flag, skip the rest of its work and
 * return.  This call synchronises the device, writes the flag to *flags_out
 * (0: no wait has expired since the last call) and clears it.  The thesis has
 * no counterpart; the outputs of a launch that set the flag are invalid. */
int dd_device_status(int* flags_out);

#ifdef __cplusplus
}
#endif

#endif /* DD_WILSON_H */
