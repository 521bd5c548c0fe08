/*
 * mpclinear.h -- C ABI of the GB300 library for one party's online
 * computation of an actively secure SPDZ2k linear layer Z = X . W with
 * CompactTag (arXiv 2311.04406).
 *
 * Notation (§2.2, §2.5): the layer multiplies X (M x K) by W (K x N).  Party i
 * holds authenticated shares of a Beaver matrix triple (A, B, C = A.B), of a
 * random mask R (M x N), their tag shares m(A), m(B), m(C), m(R), and a key
 * share alpha_i.  The public opened matrices are E = X - A (M x K) and
 * F = W - B (K x N) (the paper calls F "U"), and, for CompactTag, the opened
 * D~ = sum_i ([R]_i - [Z]_i) (M x N) and the public combiners chi (N) and
 * chi^ (M).  Party index 0 is the paper's P1.
 *
 * Memory: every matrix/vector pointer is DEVICE memory owned by the caller,
 * row-major, contiguous, 16-byte aligned, `ring.words` little-endian uint64
 * words per element (Z_2^64: one word; Z_2^128: (lo, hi)).  The library never
 * allocates or frees: scratch comes from the caller's workspace, sized by
 * mpc_workspace_size().  All calls are asynchronous on `stream` (a
 * cudaStream_t passed as void*; NULL = the legacy default stream) and return
 * after enqueueing.  Arguments are validated on the host before any launch;
 * invalid arguments return a negative status and launch nothing.  The library
 * holds no state between calls.
 *
 * All arithmetic is exact wrapping integer arithmetic mod 2^(k+s); results are
 * bit-identical for every launch configuration.
 */
#ifndef MPCLINEAR_H
#define MPCLINEAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Ring parameters (§4.1): (k, s, words) = (32, 32, 1) for Z_2^64 or
 * (64, 64, 2) for Z_2^128.  k + s must equal 64 * words. */
typedef struct {
    int32_t k;
    int32_t s;
    int32_t words;
} mpc_ring;

/* One linear layer for one party.  M, K, N >= 0 (zero-sized layers are valid
 * no-ops; K = 0 gives Z = C).  party in [0, nparties). */
typedef struct {
    int64_t M;
    int64_t K;
    int64_t N;
    mpc_ring ring;
    int32_t party;
    int32_t nparties;
} mpc_layer;

typedef enum { MPC_TAG_FULL = 0, MPC_TAG_COMPACT = 1, MPC_TAG_COMPACT_TRUNC = 2 } mpc_tag_mode;
typedef enum {
    MPC_CHECK_COMPACT = 0,
    MPC_CHECK_BATCHREC = 1,
    MPC_CHECK_BATCHREC_SEEDED = 2
} mpc_check_mode;

/* `which` argument of mpc_workspace_size */
enum {
    MPC_WS_SHARE = 0,
    MPC_WS_TAG_FULL = 1,
    MPC_WS_TAG_COMPACT = 2,
    MPC_WS_CHECK_COMPACT = 3,
    MPC_WS_CHECK_BATCHREC = 4,
    MPC_WS_PUBLIC_PRODUCT = 5,
    MPC_WS_OPTMAC_TRUNC = 6,
    MPC_WS_SHARE_TRUNC = 7
};

/* Status codes */
#define MPC_OK 0
#define MPC_E_NULL (-1)        /* a required pointer is NULL */
#define MPC_E_SHAPE (-2)       /* negative or too large M, K, N */
#define MPC_E_RING (-3)        /* unsupported (k, s, words) */
#define MPC_E_ALIGN (-4)       /* a pointer is not 16-byte aligned */
#define MPC_E_WORKSPACE (-5)   /* workspace NULL or smaller than required */
#define MPC_E_CUDA (-6)        /* a CUDA launch or runtime error */
#define MPC_E_MODE (-7)        /* unknown tag/check mode */
#define MPC_E_PARTY (-8)       /* party index outside [0, nparties) */
#define MPC_E_TIMEOUT (-9)     /* a device-side wait gave up (status read back) */
#define MPC_E_SCRATCH_LIMIT (-10) /* layer needs more than MPC_NOALLOC_SCRATCH_BYTES */
#define MPC_E_IO (-11)         /* an autotune table file could not be read or written */

/*
 * a1. Share of Z = X . W from the triple, Eq. (compute-z) and Fig. Pi_MatMul
 * steps 2-3 (§2.5):
 *     Z_i = C_i + E . B_i + A_i . F   (+ E . F when layer->party == 0)
 * E: M x K, F: K x N, A_i: M x K, B_i: K x N, C_i: M x N, Z_i: M x N (output,
 * may not alias an input).
 */
int mpc_linear_share(const mpc_layer *layer,
                     const uint64_t *E, const uint64_t *F,
                     const uint64_t *A_i, const uint64_t *B_i, const uint64_t *C_i,
                     uint64_t *Z_i,
                     void *workspace, size_t ws_bytes, void *stream);

/*
 * Tag share of Z for party i.
 *
 * MPC_TAG_FULL -- a2, the SPDZ2k recurrence, Eq. (compute-ztag) (§2.5), with
 * the alpha term added by every party:
 *     mZ_i = mC_i + E . mB_i + mA_i . F + alpha_i * (E . F)
 *   reads E, F, mA_i (M x K), mB_i (K x N), mC_i (M x N); writes mZ_i (M x N).
 *   mR_i, Dtilde, chi, mDc_i, Dc are ignored (may be NULL).
 *
 * MPC_TAG_COMPACT -- CompactTag, §3.2-§3.3 and Fig. Pi_CompactMatMul
 * steps 6-7 (untruncated layer):
 *   a3 optimistic tag (Fig. Pi_OptMAC):  mZ_i = mR_i - alpha_i * Dtilde
 *   a4 compressions (Fig. Pi_Compress): mR_i.chi, Dtilde.chi, mC_i.chi (M),
 *                                        mB_i.chi, F.chi (K)
 *   a5 compact tag, Eq. (compute-zcomptag):
 *       mZc_i = mC_i.chi + E.(mB_i.chi) + mA_i.(F.chi) + alpha_i * E.(F.chi)
 *       mDc_i = mR_i.chi - mZc_i               (output, M)
 *       Dc    = Dtilde.chi                     (output, M; the compressed D)
 *   reads E, F, mA_i, mB_i, mC_i, mR_i (M x N), Dtilde (M x N), chi (N).
 *
 * MPC_TAG_COMPACT_TRUNC -- the compact tag of the truncated layer,
 * Fig. Pi_CompactMatMul steps 6-7 (§3.4.2): as MPC_TAG_COMPACT but without
 * the E.(F.chi) term (the public E.U enters after truncation), and the
 * per-element tag comes from mpc_optmac_trunc instead: mZ_i may be NULL, in
 * which case it is not written.  mR_i is the tag share of the untruncated R.
 *
 * alpha_i: device pointer to one ring element (the key share, §2.4).
 */
int mpc_linear_tag(const mpc_layer *layer, int mode, const uint64_t *alpha_i,
                   const uint64_t *E, const uint64_t *F,
                   const uint64_t *mA_i, const uint64_t *mB_i, const uint64_t *mC_i,
                   const uint64_t *mR_i, const uint64_t *Dtilde, const uint64_t *chi,
                   uint64_t *mZ_i, uint64_t *mDc_i, uint64_t *Dc,
                   void *workspace, size_t ws_bytes, void *stream);

/*
 * a6. Check share of party i, written to cs_i (device, one ring element).
 *
 * MPC_CHECK_COMPACT -- Fig. Pi_CompactMatMul verification steps 3-5, reduced
 * mod 2^(k+s):  cs_i = sum_r chi_hat_r * (alpha_i * Dc_r - mDc_i_r)
 *   chi_hat: M, opened = Dc: M, tag_i = mDc_i: M.  Parties accept iff the sum
 *   of all cs_i is 0 mod 2^(k+s).
 * MPC_CHECK_BATCHREC -- tag check of Fig. Pi_BatchRec (§2.5) steps 2-3:
 *   cs_i = sum_{p,q} chi_pq * (mW_i_pq - alpha_i * W_pq)
 *   chi_hat = chi: M x N, opened = W: M x N, tag_i = mW_i: M x N.
 * MPC_CHECK_BATCHREC_SEEDED -- the same check with the combiners expanded
 *   from a public coin-tossed seed (F_Rand, App. A.1) instead of stored:
 *   chi_hat points to ONE 64-bit word, the seed, in device memory, and
 *   chi_pq (row-major index i = p N + q) = SplitMix64 output i of the sequence
 *   whose state starts at the seed, mod 2^s (s = layer->ring.s <= 64):
 *     chi_i = mix(seed + (i + 1) * 0x9E3779B97F4A7C15),
 *     mix(z) = ((z ^ z>>30) * 0xBF58476D1CE4E5B9 -> z ^ z>>27) * 0x94D049BB133111EB -> z ^ z>>31.
 *   The check then reads only W and mW_i.
 * The BATCHREC modes use a workspace (MPC_WS_CHECK_BATCHREC).
 */
int mpc_tag_check(const mpc_layer *layer, int mode, const uint64_t *alpha_i,
                  const uint64_t *chi_hat, const uint64_t *opened,
                  const uint64_t *tag_i, uint64_t *cs_i,
                  void *workspace, size_t ws_bytes, void *stream);

/*
 * Grouped calls: many layers in one call (a whole network's linear layers,
 * or many requests' layers).  Same results, bit for bit, as calling
 * mpc_linear_share / mpc_linear_tag once per layer in order.  The paper runs
 * its layers one at a time; grouping exists so that small layers share the
 * GPU: every tensor-core layer of the group (up to 64 per launch) is scheduled
 * by ONE persistent prologue + GEMM launch pair whose CTAs work through the
 * layers' (tile, K interval) units in turn; the remaining layers run the
 * integer-pipe kernels on side streams of the library, concurrently with one
 * another and with that launch pair (forked from and joined back to `stream`
 * with events, so the call stays ordered on `stream` and can be captured).
 * A tensor-core layer long enough to keep every SM busy for 64 waves of units
 * gets a launch pair of its own (it gains nothing from sharing one and runs
 * faster alone).
 *
 * layers[count], ptrs[count]: HOST arrays, read during the call only.  All
 * layers share one ring (MPC_E_RING otherwise); the party may differ per
 * layer.  No output may overlap any input or output of another layer of the
 * group (the layers run concurrently).  workspace: 256-byte aligned,
 * mpc_workspace_size_grouped(layers, count, which) bytes.
 */
typedef struct {
    const uint64_t *E, *F, *A_i, *B_i, *C_i;
    uint64_t *Z_i;
} mpc_share_ptrs;

typedef struct {
    const uint64_t *alpha_i, *E, *F, *mA_i, *mB_i, *mC_i, *mR_i, *Dtilde, *chi;
    uint64_t *mZ_i, *mDc_i, *Dc;
} mpc_tag_ptrs;

int mpc_linear_share_grouped(const mpc_layer *layers, int count, const mpc_share_ptrs *ptrs,
                             void *workspace, size_t ws_bytes, void *stream);

/* mode: MPC_TAG_FULL, MPC_TAG_COMPACT or MPC_TAG_COMPACT_TRUNC, as in
 * mpc_linear_tag, for every layer of the group. */
int mpc_linear_tag_grouped(const mpc_layer *layers, int count, int mode, const mpc_tag_ptrs *ptrs,
                           void *workspace, size_t ws_bytes, void *stream);

/* which: MPC_WS_SHARE, MPC_WS_TAG_FULL or MPC_WS_TAG_COMPACT.  0 on invalid
 * arguments (as mpc_workspace_size). */
size_t mpc_workspace_size_grouped(const mpc_layer *layers, int count, int which);

/*
 * a6 for many layers at once: the compact check share of each layer, exactly
 * as mpc_tag_check(layer, MPC_CHECK_COMPACT, ...) computes it (Fig.
 * Pi_CompactMatMul verification steps 3-5, reduced mod 2^(k+s)):
 *     cs_i = sum_r chi^_r (alpha_i Dc_r - mDc_{i,r}),  r < M of that layer.
 * layers[count], ptrs[count]: HOST arrays read during the call; every layer
 * in one ring (MPC_E_RING otherwise); per layer alpha_i (1 element), chi_hat,
 * Dc, mDc_i (M elements) and cs_i (1 element, output) are device pointers,
 * 16-byte aligned.  One kernel per 64 layers, no workspace.  Batching only:
 * the paper checks layer by layer.
 */
typedef struct {
    const uint64_t *alpha_i, *chi_hat, *Dc, *mDc_i;
    uint64_t *cs_i;
} mpc_check_ptrs;

int mpc_tag_check_grouped(const mpc_layer *layers, int count, const mpc_check_ptrs *ptrs, void *stream);

/* Kernels one grouped call enqueues (which as above); negative on invalid
 * arguments. */
int mpc_launch_count_grouped(const mpc_layer *layers, int count, int which);

/*
 * Launch table (autotuner).  The paper has no counterpart: every GEMM path of
 * this library computes the same exact sums, so the choice of path and tile
 * shape is a matter of speed only.  For each layer shape (ring width, M, K, N)
 * the table holds a choice -- path 1, the tensor-core kernel, with output
 * tiles of `tile_rows` rows: 128; 64 (an M = 64 MMA takes as long as an
 * M = 128 one, so the 64-row tile halves only the shared-memory bytes of the
 * left operand); or the wide tile, tile_rows = 32 for Z_2^64 and 16 for
 * Z_2^128, which puts 128 output columns on the tensor core's M side and that
 * many of the layer's rows on its N side (for layers with few rows); or the
 * tall tile, tile_rows = -128: 128-row tiles whose left operand [E | X] the
 * GEMM turns into digit planes itself, with the c E term moved to the right
 * operand ([E | X + cE].[B ; F] = [E | X].[B + cF ; F]), so that no digit
 * plane of the left operand goes through memory (for tall, narrow layers;
 * needs K words even for the 2-D loads) -- and
 * `swizzle` tiles per tile-order group (1-64); or path 0, the integer-pipe kernels, with tiles
 * of `tile_rows` rows (64 or 16; 0 = 16 when 64-row tiles would give fewer
 * blocks than SMs, else 64; skinny layers with M <= 8 use a GEMV whatever the
 * value) and a K-split target of `waves` x 152 blocks (0 = default).  Untuned
 * shapes use a built-in rule (tensor cores from 2^22 ring MACs, 2^20 for
 * Z_2^128; the wide tile up to two of its row tiles, and for Z_2^128 up to
 * M = 64 when it has a work unit per SM; 64-row tiles up to M = 64, the tall tile for layers with N <= 64 and M >= 2048 (Z_2^64) or
 * M >= 1024 (Z_2^128), and for N <= 128 from M = 4096).  The table is process-wide and thread-safe; workspace
 * sizes do not depend on it.
 *
 * mpc_autotune: for each distinct shape of layers[count], times the
 *   candidates (128-row tiles, 64-row tiles for M <= 64, the wide tile for
 *   M <= 128, the tall tile for M >= 128, each with swizzle 1/4/8/16 on the
 *   tensor cores; tile heights 64 and 16 with K-split 1/2/4/8
 *   on the integer pipes, below 2^31 ring MACs) on `stream` and stores the
 *   fastest.  Synchronous;
 *   allocates and frees its own scratch operands; do not call it during
 *   stream capture.  Returns the number of shapes tuned, or a status.
 * mpc_autotune_set: store a choice (MPC_E_MODE if the tensor-core kernel
 *   cannot run the shape with that tile height, or a value is out of range).
 * mpc_autotune_choice: the choice a call would use now; returns 1 if it comes
 *   from the table, 0 for the built-in rule.
 * mpc_autotune_save / _load: the table as text ("mpclinear-autotune 2", then
 *   "words M K N path tile_rows swizzle waves" per line; version-1 files
 *   without tile_rows load as 128-row tiles); return the number of shapes, or
 *   MPC_E_IO.  Loading merges into the table.
 * mpc_autotune_clear: empties the table; returns the number of shapes removed.
 */
int mpc_autotune(const mpc_layer *layers, int count, void *stream);
int mpc_autotune_set(const mpc_layer *layer, int path, int tile_rows, int swizzle, int waves);
int mpc_autotune_choice(const mpc_layer *layer, int *path, int *tile_rows, int *swizzle, int *waves);
int mpc_autotune_save(const char *path);
int mpc_autotune_load(const char *path);
int mpc_autotune_clear(void);

/*
 * Allocation-free variant of mpc_linear_tag(layer, MPC_TAG_COMPACT, ...).  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory -- e.g. a host runtime reaching this library through
 * a plain C FFI with no CUDA allocator of its own, or a serving process whose
 * device memory is wholly owned by another framework's pool -- and so cannot
 * pass a workspace.  Same arguments, results and layouts as the COMPACT tag
 * call, minus the workspace.
 *
 * Scratch comes from one static device array of MPC_NOALLOC_SCRATCH_BYTES
 * (4 MiB) that every GPU loading this library holds until the process exits.
 * Layers whose mpc_workspace_size(layer, MPC_WS_TAG_COMPACT) exceeds it are
 * rejected with MPC_E_SCRATCH_LIMIT before any launch.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  All calls share the array:
 * calls whose kernels overlap on the GPU (unordered streams) race, so order
 * them.  Nothing in this call allocates or frees memory.
 */
#define MPC_NOALLOC_SCRATCH_BYTES (4u << 20)
int mpc_linear_tag_compact_noalloc(const mpc_layer *layer, const uint64_t *alpha_i,
                                   const uint64_t *E, const uint64_t *F,
                                   const uint64_t *mA_i, const uint64_t *mB_i,
                                   const uint64_t *mC_i, const uint64_t *mR_i,
                                   const uint64_t *Dtilde, const uint64_t *chi,
                                   uint64_t *mZ_i, uint64_t *mDc_i, uint64_t *Dc,
                                   void *stream);

/*
 * Pi_BatchRec open phase step 1 (§2.5) for an opened difference V = X - A
 * (E = X - A or U = Y - B, Fig. Pi_MatMul step 1), rows x cols elements:
 *   W_i = X_i - A_i + R_i,   mW_i = mX_i - mA_i + mR_i
 * R_i, mR_i: shares of a mask that is 0 mod 2^k and of its tag (so the opened
 * W equals V mod 2^k while its top s bits are masked).  A_i and mA_i may be
 * NULL (V = X).  W_i is the share each party broadcasts; mW_i is kept for the
 * tag check (mpc_tag_check BATCHREC modes).  No workspace.
 */
int mpc_batchrec_mask(const mpc_ring *ring, int64_t rows, int64_t cols,
                      const uint64_t *X_i, const uint64_t *A_i, const uint64_t *R_i,
                      const uint64_t *mX_i, const uint64_t *mA_i, const uint64_t *mR_i,
                      uint64_t *W_i, uint64_t *mW_i, void *stream);

/*
 * Linear combination of ring arrays, out = sum_j coef[j] * in[j] mod 2^(k+s),
 * elementwise over n elements, 1 <= count <= 16, coef[] small signed integers
 * (host array), in[] a host array of device pointers.  Authenticated shares are
 * linear under public constants (§2.4), so this is the local part of an
 * opening when several parties are simulated on one device (E = sum_i
 * (X_i - A_i), Fig. Pi_MatMul step 1; D~ = sum_i (R_i - Z_i), Fig. Pi_OptMAC)
 * and of the mask arithmetic around it.  out may alias an input (each element
 * is read before it is written by the same thread).  No workspace.
 */
int mpc_lincomb(const mpc_ring *ring, int64_t n, int count, const int64_t *coef,
                const uint64_t *const *in, uint64_t *out, void *stream);

/* `groups` linear combinations with the same coefficients in one launch per
 * 64 groups: out[g] = sum_j coef[j] * in[g * count + j] over n[g] elements
 * (1 <= count <= 4; n, in and out are host arrays of sizes and device
 * pointers).  The arithmetic of mpc_lincomb for each group; the groups must
 * not overlap one another's outputs (they run concurrently).  No workspace. */
int mpc_lincomb_grouped(const mpc_ring *ring, int groups, const int64_t *n, int count, const int64_t *coef,
                        const uint64_t *const *in, uint64_t *const *out, void *stream);

/*
 * im2col view of a convolution (§2.6): for a batch of `channels` x height x
 * width images in NCHW layout and an f x f filter with zero padding `pad`
 * (< f) and stride `stride`, out is the (batch H' W') x (channels f f) matrix
 * with H' = (height - f + 2 pad) / stride + 1 (floor; the textbook size, see
 * the "+1" reading of §2.6), W' likewise: row (b, oy, ox), column (c, ky, kx)
 * holds in[b][c][oy stride + ky - pad][ox stride + kx - pad], or 0 in the
 * padding.  The convolution with a (channels f f) x out_channels weight is
 * then the ring GEMM of mpc_linear_share.  Local and linear: each party applies
 * it to its shares and tags.  MPC_E_SHAPE for f < 1, pad >= f, stride < 1 or
 * an image smaller than the filter.  No workspace.
 */
int mpc_im2col(const mpc_ring *ring, int64_t batch, int64_t channels, int64_t height, int64_t width,
               int f, int pad, int stride, const uint64_t *in, uint64_t *out, void *stream);

/*
 * Local transpose, out (cols x rows) = in (rows x cols)^T.  Training's
 * backward linear layers (§4: grad X = grad Z . W^T, grad W = X^T . grad Z) are
 * the same per-party Beaver products on transposed operands; shares and tags
 * transpose locally (the transpose of a sharing is a sharing of the
 * transpose, §2.4 linearity).  in and out must not overlap.  No workspace.
 */
int mpc_transpose(const mpc_ring *ring, int64_t rows, int64_t cols,
                  const uint64_t *in, uint64_t *out, void *stream);

/*
 * Truncated layer (Fig. Pi_CompactMatMul with Fig. Pi_OptMAC&Trunc, §3.4).
 *
 * mpc_linear_share_trunc -- step 2: Z_i = C_i + E . B_i + A_i . F for every
 *   party, party 0 included (no E . F: the public product is added after
 *   truncation).  Arguments and layouts as mpc_linear_share; workspace
 *   MPC_WS_SHARE_TRUNC.
 *
 * mpc_public_product -- P = E . F (M x N), the public product every party
 *   computes from the opened matrices.  Workspace MPC_WS_PUBLIC_PRODUCT.
 *
 * mpc_optmac_trunc -- steps 3-4 (Pi_OptMAC&Trunc steps 3-4 plus P1's public
 *   term), elementwise over M x N:
 *     delta = (Dtilde mod 2^k) / 2^f,  rho = (P mod 2^k) / 2^f  (floor),
 *     tau = rho - delta,
 *     Zf_i  = Rf_i  + tau          (party 0 only; others copy Rf_i)
 *     mZf_i = mRf_i + alpha_i tau  (every party)
 *   Rf_i, mRf_i: shares of R^f = R / 2^f and of its tag; Dtilde: the opened
 *   D~ = sum_j (R_j - Z_j); P from mpc_public_product.  0 <= f <= k
 *   (MPC_E_SHAPE otherwise).  No workspace.
 */
int mpc_linear_share_trunc(const mpc_layer *layer,
                           const uint64_t *E, const uint64_t *F,
                           const uint64_t *A_i, const uint64_t *B_i, const uint64_t *C_i,
                           uint64_t *Z_i,
                           void *workspace, size_t ws_bytes, void *stream);

int mpc_public_product(const mpc_layer *layer, const uint64_t *E, const uint64_t *F,
                       uint64_t *P, void *workspace, size_t ws_bytes, void *stream);

int mpc_optmac_trunc(const mpc_layer *layer, int f, const uint64_t *alpha_i,
                     const uint64_t *Rf_i, const uint64_t *mRf_i, const uint64_t *Dtilde,
                     const uint64_t *P, uint64_t *Zf_i, uint64_t *mZf_i, void *stream);

/* Bytes of workspace the call `which` (MPC_WS_*) needs for this layer; 0 for
 * an invalid layer.  A larger workspace is always accepted. */
size_t mpc_workspace_size(const mpc_layer *layer, int which);

/* Which ring-GEMM kernel mpc_linear_share / MPC_TAG_FULL use for this layer:
 * 1 = the tensor-core kernel, 0 = the integer-pipe kernel, negative = invalid
 * layer (status code).  Pure host query; launches nothing. */
int mpc_gemm_path(const mpc_layer *layer);

/* Number of kernels the call `which` (MPC_WS_* numbering) enqueues for this
 * layer (0 for empty layers); negative status for an invalid layer.  Pure
 * host query. */
int mpc_launch_count(const mpc_layer *layer, int which);

/* Reads and clears the device flag that a kernel sets when one of its bounded
 * waits gave up (so that it returned instead of hanging; its outputs are then
 * wrong).  The read runs on a private non-blocking stream of the library and
 * returns when it is done: it neither waits for nor orders itself with the
 * caller's streams, so a kernel still running may set the flag after the read
 * (the next query reports it).  To cover a given call, query after that call
 * has completed.  Returns MPC_E_TIMEOUT if the flag was set since the last
 * query, MPC_OK if not, MPC_E_CUDA if it could not be read.  Uses the current
 * device. */
int mpc_device_status(void);

/* Self-test of the bounded device-side wait (no counterpart in the paper):
 * one thread waits on a barrier that nothing arrives at, for at most
 * limit_cycles clock cycles (1e3 .. 1e10; about 1e9 per 0.5 s at 2 GHz), then
 * gives up and records the timeout as the GEMM's roles do.  Synchronous on
 * `stream`.  Returns MPC_E_TIMEOUT when the wait gave up (the expected
 * outcome; the flag that mpc_device_status reads is then set), MPC_OK if it did
 * not, MPC_E_SHAPE for a limit out of range, MPC_E_CUDA on a CUDA error.  The
 * context stays usable afterwards. */
int mpc_selftest_wait(long long limit_cycles, void *stream);

/* Static string for a status code. */
const char *mpc_status_str(int status);

/* Library ABI version (major * 100 + minor). */
int mpc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MPCLINEAR_H */
