/*
 * abft.h -- C ABI of libabft: Huang-Abraham algorithm-based fault-tolerant
 * matrix multiplication on one NVIDIA GB300 (sm_103a).
 *
 * Method: Bosilca, Delmas, Dongarra, Langou, "Algorithmic Based Fault
 * Tolerance Applied to High Performance Computing" (2008).  A is extended with
 * checksum rows C_C^T A, B with checksum columns B C_R, and the product of the
 * extended operands is the full-checksum matrix (AB)_F (section 2.2, Eq. (1)).
 * Its consistency detects, locates and corrects a corrupted element of C, and
 * a block checksum rebuilds a lost block (section 2.1).
 *
 * Conventions shared by every entry point
 *  - Matrices are row-major; lda/ldb/ldc are leading dimensions in elements.
 *    C = A B with A m-by-k, B k-by-n, C m-by-n.
 *  - Pointers named A, B, C, ws, a_scale, b_scale are DEVICE pointers, owned by
 *    the caller, who keeps them alive until the stream work completes.  Host
 *    pointers are marked (host).  The library allocates no device memory per
 *    call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are stream-ordered and asynchronous unless stated otherwise: work
 *    that produced the inputs or the workspace on another stream must be
 *    ordered before the call by the caller (an event or a stream wait; a
 *    non-blocking stream does not wait for the legacy default stream).
 *  - No C++ exception crosses the ABI.  Every call returns an abft_status; on a
 *    non-OK status abft_last_error() (thread-local) holds a one-line message.
 *    An invalid descriptor or argument returns ABFT_ERR_INVALID with nothing
 *    launched.
 *  - Verify blocks: rows of C are cut into blocks of vb_rows rows and columns
 *    into blocks of vb_cols columns (the last ones may be shorter).  Each block
 *    has an unweighted checksum (weights 1) and a weighted checksum with
 *    weights w_t = (t+1) * 2^-ceil(log2 vb) for the t-th row (column) of the
 *    block; the power-of-two scale is exact and keeps weighted sums in range.
 *  - Erasure grid: grid_p x grid_q blocks (m % grid_p == 0, n % grid_q == 0).
 *    A also gains m/grid_p block checksum rows S_A = sum_I A_I, so the product
 *    carries S = sum_I C_I, enough to rebuild one lost block per block column.
 *  - Workspaces (ws) are 256-byte aligned device buffers (see
 *    abft_workspace_bytes).
 *
 * Environment variables read at each launch (tuning and testing only; the
 * defaults are the measured best choices):
 *  - ABFT_PROMOTE_KSTEPS  tensor-core k-steps (64 wide) accumulated before the
 *                         epilogue adds a partial into fp32 registers (0: none;
 *                         default 8 for ABFT_BF16X6, 16 for ABFT_BF16X3, 0 else).
 *  - ABFT_TALL_TILES      0 / 1: 128- or 256-row tiles for products without
 *                         promotion (default: 256 rows when m > 128 and the K
 *                         loop has at least 32 k-steps).
 *  - ABFT_PAIR_TILES      1: single products run 256 x 256 tiles on CTA pairs
 *                         (clusters of two, one cta_group::2 MMA per K step;
 *                         default 0: one-CTA tiles, see ABFT_TALL_TILES).
 *  - ABFT_GROUP_M         raster group height in tile rows of single products
 *                         (default 2048 rows).
 *  - ABFT_GRP_SWAP        0: grouped products compute checksum rows in regular
 *                         tiles instead of swapped ones (default 1).
 *  - ABFT_TUNE_CACHE      file of grouped-product tunings (abft_group_autotune).
 *  - ABFT_FP8_NATIVE      0: ABFT_FP8_E4M3 data tiles multiply the dequantised
 *                         bf16 planes instead of the e4m3 codes (comparison
 *                         only; an encode and its product must see the same
 *                         value).
 *  - ABFT_FP8_CS_STRIDE   position stride of the checksum tiles in the FP8
 *                         product's tile order (default 1: all first).
 *  - ABFT_TEST_STALL_PRODUCER  1: the tensor-core product's producer skips its
 *                         first tile so its bounded waits run out (tests of
 *                         ABFT_ERR_TIMEOUT; never set in production).
 */
#ifndef ABFT_H
#define ABFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ABFT_OK = 0,
  ABFT_ERR_INVALID = 1,       /* bad descriptor / argument; nothing launched */
  ABFT_ERR_CUDA = 2,          /* a CUDA call failed; see abft_last_error()   */
  ABFT_ERR_UNSUPPORTED = 3,   /* valid request this build does not provide   */
  ABFT_ERR_UNCORRECTABLE = 4, /* errors found that could not all be fixed    */
  ABFT_ERR_TIMEOUT = 5        /* a bounded device wait gave up               */
} abft_status;

typedef enum {
  ABFT_F64 = 0,     /* A, B, C binary64; DFMA product, binary64 checksums          */
  ABFT_BF16 = 1,    /* A, B bfloat16; C binary32; tensor-core product, fp32 accum.  */
  ABFT_BF16X3 = 2,  /* A, B binary32 split into bf16 hi+lo planes by abft_encode;
                       product A_hi B_hi + A_hi B_lo + A_lo B_hi; C binary32        */
  ABFT_FP8_E4M3 = 3, /* A, B e4m3 with binary32 scales per 128x128 block; C binary32 */
  ABFT_BF16X6 = 4   /* A, B binary32 split into three bf16 planes (x = p0 + p1 + p2,
                       24 significant bits) by abft_encode; the six products
                       p_a q_b with a + b <= 2; C binary32 (fp32-level accuracy)    */
} abft_dtype;

/* Report kinds (abft_fault.kind). */
#define ABFT_KIND_CORRECTED 1          /* located by the checksums and recomputed */
#define ABFT_KIND_NONFINITE_CORRECTED 2 /* a NaN/Inf element located and recomputed */
#define ABFT_KIND_UNCORRECTABLE 3      /* a flagged line that could not be fixed   */
#define ABFT_KIND_BLOCK_RECOVERED 4    /* an erased block rebuilt                  */

typedef struct {
  int64_t m, n, k;       /* C = A B: A m-by-k, B k-by-n                             */
  int64_t lda, ldb, ldc; /* leading dimensions in elements (>= k, n, n)            */
  int32_t dtype;         /* abft_dtype                                             */
  int32_t vb_rows;       /* verify block rows (1 .. m)                             */
  int32_t vb_cols;       /* verify block columns (1 .. n)                          */
  int32_t grid_p;        /* erasure grid block-rows; 0 = no block checksum         */
  int32_t grid_q;        /* erasure grid block-columns (with grid_p > 0)           */
  int32_t flags;         /* reserved, must be 0                                    */
  double tau_safety;     /* safety factor s of the detection threshold; 0 -> 4     */
  int32_t grid_f;        /* block checksums of the erasure grid, 1..4 (0 -> 1): up
                            to grid_f erased blocks per block column are rebuilt  */
  int32_t reserved;      /* must be 0                                              */
} abft_desc;

/* One report entry.  row/col are element coordinates; -1 marks the unknown
 * coordinate of a flagged line (col = -1: row check of row `row`; row = -1:
 * column check of column `col`).  side: 0 column check, 1 row check, 2 erasure.
 * delta = value before - value after correction; r_e / r_w are the unweighted
 * and weighted residuals of the line that located it.  problem is the index of
 * the problem in a group (abft_group_*), 0 for the single-problem calls. */
typedef struct {
  int32_t row, col, kind, side;
  double delta, r_e, r_w;
  int32_t problem, reserved;
} abft_fault;

/* Byte offsets of the regions inside the workspace (all 256-byte aligned) and
 * their shapes, for callers that want to read the checksums.  R = 2*nvr + bs
 * checksum rows (nvr = ceil(m/vb_rows), bs = m/grid_p or 0), Cc = 2*nvc
 * checksum columns (nvc = ceil(n/vb_cols)).  acs (acs_rows x acs_ld) and bcs
 * (k x bcs_ld, row-major) hold the encoded operand rows/columns in the
 * product's operand format: binary64 for ABFT_F64 (acs_rows = R, bcs_cols =
 * Cc); for the tensor-core dtypes every fp32 checksum is a bf16 hi + lo pair
 * (acs_rows = 4*nvr + 2*bs, bcs_cols = 4*nvc) whose products land in E16 / F16
 * (fp32) and are summed in binary64.  E (R-by-n binary64) holds the expected
 * column checksums of each verify block (unweighted, weighted), then the
 * block checksum rows S; F (m-by-Cc binary64) the expected row checksums. */
typedef struct {
  size_t total;
  size_t acs, bcs, E, F;
  size_t nArow, nAblk, nBcol, nBblk; /* threshold norms (binary64)             */
  size_t scratch, scratch_bytes;     /* verify lists, counters, report buffer */
  int64_t R, Cc, nvr, nvc, bs;
  int64_t acs_ld, bcs_ld;            /* leading dims of acs / bcs in elements  */
  size_t E16, F16;                   /* fp32 product rows/columns of the bf16
                                        checksum pieces (tensor-core dtypes)  */
  int64_t acs_rows, bcs_cols;        /* rows of acs, columns of bcs            */
  size_t obs_col, obs_row;           /* fused observed partial sums (fp32)     */
  size_t inject;                     /* armed epilogue fault injections        */
  int32_t fused;                     /* 1: abft_gemm writes observed sums      */
  int32_t planes;                    /* bf16 planes per operand: 2 for BF16X3,
                                        3 for BF16X6, else 1                   */
  size_t acs_plane, bcs_plane;       /* bytes from one plane to the next       */
  size_t op_a, op_b;                 /* split dtypes: the planes of A and B
                                        (op_a_ld apart by align256 of a plane);
                                        FP8: the dequantised bf16 operands     */
  int64_t op_a_ld, op_b_ld;          /* their leading dims (elements)          */
  size_t car_a, car_b;               /* chained calls: bounds of the carried
                                        checksums' deviation (binary64, 2 per
                                        row / column verify block; zero after
                                        abft_encode)                           */
  size_t scales;                     /* FP8: the block scales of A, then of B
                                        (binary32, copied by abft_encode)      */
  size_t f8grp;                      /* FP8: scale groups of the product's data
                                        tiles (written by abft_gemm)           */
  size_t f8bt;                       /* FP8: B's e4m3 codes transposed (n rows
                                        of ceil16(k) bytes, by abft_encode)    */
} abft_ws_layout;

/* Size of the caller-owned device workspace for `desc`.  Returns 0 for an
 * invalid descriptor (abft_last_error() says why).  Every call that takes a
 * workspace requires its base to be 256-byte aligned (cudaMalloc and the
 * PyTorch caching allocator give at least that) and returns ABFT_ERR_INVALID
 * with nothing launched otherwise. */
size_t abft_workspace_bytes(const abft_desc* desc);

/* Fill *out (host) with the workspace layout.  ABFT_ERR_INVALID on a bad desc. */
abft_status abft_workspace_layout(const abft_desc* desc, abft_ws_layout* out);

/* Checksum encoding (section 2.1; the operands of Eq. (1)).  Writes into ws the
 * checksum rows of A (per verify block: e^T A_I and w^T A_I; then S_A when the
 * erasure grid is on) and the checksum columns of B (B_J e, B_J w), plus the
 * norms the detection thresholds use.  a_scale/b_scale: binary32 block scales
 * for ABFT_FP8_E4M3 (ceil(m/128) x ceil(k/128) and ceil(k/128) x ceil(n/128),
 * row-major), else NULL.  ABFT_FP8_E4M3: A and B are e4m3 bytes (lda, ldb in
 * elements); the scales must be powers of two, 2^e with -117 <= e <= 119 (or
 * zero), so that every dequantised value e4m3(q) * scale is exact in bf16 --
 * the encode writes those values as bf16 operand planes into ws and forms the
 * checksums from them (a scale outside that set, or a NaN code, sets a status
 * word of this workspace, and abft_verify_correct on it returns
 * ABFT_ERR_INVALID until the next encode).  When A and B have
 * 16-byte aligned rows (base and lda, ldb multiples of 16) the encode also
 * copies the scales, writes B's codes transposed (layout.f8bt) and the scale
 * groups of the product's data tiles (layout.f8grp), for the product's FP8
 * tensor-core data tiles.  Asynchronous. */
abft_status abft_encode(const abft_desc* desc, const void* A, const void* B, const void* a_scale,
                        const void* b_scale, void* ws, void* stream);

/* abft_encode for callers that cannot allocate device memory.  The paper has
 * no counterpart: this is an interface convenience of this library.  Some
 * callers cannot call cudaMalloc -- code that runs while a CUDA graph is being
 * captured, real-time or signal-context threads that must not take the
 * allocator's lock, or plugins that only receive buffers from their host
 * application.  Such a caller may not be able to size a workspace with its
 * scratch part.  This entry point writes the same outputs as abft_encode into
 * ws, but ws only needs the bytes below abft_ws_layout.scratch: the encode's
 * partial sums go to an 8 MiB array of static device memory inside the
 * library, which each device that loads the library keeps until the process
 * exits.  It allocates nothing.  Problems whose partial sums need more than
 * 8 MiB (about 8 * (k/256 * (n + 4*nvr) + k/64 * 4*nvc) bytes) return
 * ABFT_ERR_INVALID with nothing launched.  Every call looks up the array's
 * device address on the current device (cudaGetSymbolAddress; nothing is
 * cached, so a device reset leaves no stale address); the first call on a
 * device may load the library's device code, so make it before any stream
 * capture.  All calls share the one array, so
 * calls that overlap on the GPU (different streams, threads) race and must be
 * serialised by the caller.  ABFT_F64 only.  Asynchronous. */
abft_status abft_encode_noalloc(const abft_desc* desc, const void* A, const void* B,
                                const void* a_scale, const void* b_scale, void* ws, void* stream);

/* Chained encode (section 3.2: ABFT BLAS calls stacked one after the other do
 * not recompute the checksums between calls).  Like abft_encode, except that
 *  - left_desc / left_ws (may be NULL): A is the output C of that earlier
 *    product, whose workspace still holds its expected checksums.  Its column
 *    checksum rows E (and its first grid_f block checksum rows) become this
 *    product's encoded rows of A; A is read only for the threshold norms.
 *    Requires left_desc->m == m, left_desc->n == k, the same vb_rows and,
 *    when this desc has an erasure grid, the same grid_p and a left grid_f of
 *    at least this grid_f.
 *  - right_desc / right_ws (may be NULL): B is the output of that earlier
 *    product; its row checksum columns F become this product's encoded
 *    columns of B.  Requires right_desc->m == k, right_desc->n == n and the
 *    same vb_cols.
 * The carried checksums differ from the sums of the stored operand by the
 * earlier products' rounding; the detection thresholds of this product gain
 * that deviation's bound (car_a / car_b in abft_ws_layout), carried on
 * through further chained calls.  Because the checksums are carried and not
 * recomputed, an operand value that changed after the earlier product's
 * verify is caught by this product's verify: the whole output row (left) or
 * column (right) it spoils is recomputed from the carried checksums, and the
 * other side's lines, whose expectations were formed from the changed
 * operand, are reported ABFT_KIND_UNCORRECTABLE (status
 * ABFT_ERR_UNCORRECTABLE; at most 2048 elements can be recomputed in one
 * verify).  dtype ABFT_F64, ABFT_BF16X3 or ABFT_BF16X6 (ABFT_ERR_UNSUPPORTED
 * otherwise).  An ABFT_F64 product chains to ABFT_F64 products (binary64 C);
 * a split product chains to any tensor-core product (binary32 C: ABFT_BF16,
 * ABFT_BF16X3, ABFT_BF16X6, ABFT_FP8_E4M3), whose binary64 checksums enter
 * its checksum planes as two (X3) or three (X6) bf16 pieces; other pairings
 * return ABFT_ERR_INVALID.  With both left and right NULL this is
 * abft_encode.  Asynchronous; the earlier workspaces must stay untouched
 * until the call completes on the stream. */
abft_status abft_encode_chained(const abft_desc* desc, const void* A, const void* B,
                                const abft_desc* left_desc, const void* left_ws,
                                const abft_desc* right_desc, const void* right_ws, void* ws,
                                void* stream);

/* The ABFT product (Eq. (1)): [A; C_C^T A] [B, B C_R] on the GPU.  Writes the
 * data block A B into C and the checksum blocks into ws (E and F).  Requires a
 * preceding abft_encode on the same ws and operands.  ABFT_BF16X3 and
 * ABFT_BF16X6 multiply the bf16 operand planes that encode wrote.
 * ABFT_FP8_E4M3: the data block multiplies the e4m3 codes of A and the
 * transposed codes of B that encode wrote, on the 8-bit tensor path
 * (tcgen05 kind::f8f6f4) with fp32 accumulation, each run of k-steps (128
 * wide) with the same block-scale product in its own accumulator, scaled once
 * by that power of two (exact); the checksum blocks multiply the bf16 planes.
 * Without 16-byte aligned rows the data block multiplies the planes too.
 * a_scale and b_scale are not read (the encode kept a copy).  Asynchronous. */
abft_status abft_gemm(const abft_desc* desc, const void* A, const void* B, const void* a_scale,
                      const void* b_scale, void* C, void* ws, void* stream);

/* Fault injection into the accumulator outputs of the tensor-core product
 * (compute faults, as opposed to abft_inject_bitflips on the stored C): arms
 * up to 256 flips (host arrays rows, cols, bits; bit 0..31 of the fp32
 * element) that every following abft_gemm on this ws applies inside its
 * epilogue, before C is stored and before the fused observed checksums are
 * formed.  count = 0 disarms.  ABFT_ERR_UNSUPPORTED for ABFT_F64.  The paper
 * injects process failures in its stress test (section 4.3); this is the
 * bit-flip analogue.  Asynchronous. */
abft_status abft_set_epilogue_faults(const abft_desc* desc, void* ws, const int64_t* rows,
                                     const int64_t* cols, const int32_t* bits, int32_t count,
                                     void* stream);

/* The same GEMM kernel with no checksum tiles: C = A B only.  This is the
 * checksum-free baseline the ABFT overhead is measured against.  ws may be
 * NULL except for ABFT_BF16X3, ABFT_BF16X6 and ABFT_FP8_E4M3, whose products read the bf16
 * operand planes a preceding abft_encode wrote into ws.  A bounded wait that
 * gives up is recorded in ws's status word (as for abft_gemm); without ws it
 * is not reported.  Asynchronous. */
abft_status abft_gemm_plain(const abft_desc* desc, const void* A, const void* B,
                            const void* a_scale, const void* b_scale, void* C, void* ws,
                            void* stream);

/* Detect, locate and correct (section 1 and section 2.2: the consistency of
 * (AB)_F detects, localizes and corrects errors in the output).  Checks every
 * column line (verify block x column) and row line (row x verify block) of C
 * against E / F, skipping lines that touch the erased blocks listed in
 * erased_blocks (host, n_erased (bi, bj) pairs).  A flagged line proposes its
 * single non-finite element or the position given by the ratio of weighted to
 * unweighted residual; each candidate is recomputed in binary64 from a line in
 * which it is the only candidate, then both its lines are checked again.
 * C is corrected in place.  reread_C: 1 re-reads all of C from memory (catches
 * faults that hit C after the product); 0 uses the observed column and row sums
 * that the tensor-core product formed in its epilogue (layout.fused = 1: bf16
 * with vb_rows a multiple of 128 and vb_cols a multiple of 32 that divides or
 * is a multiple of 256), reading C only for the lines it has to locate or
 * correct; without fused sums (ABFT_F64, other block sizes) 0 re-reads C too.  The report (host, max_reports entries) receives up to
 * max_reports entries sorted by (row, col, kind); *n_reports (host) gets the
 * full count.  SYNCHRONISES `stream`.  Returns ABFT_OK, or
 * ABFT_ERR_UNCORRECTABLE when a flagged line could not be fixed (those
 * elements are left unmodified).  ABFT_ERR_TIMEOUT, with C left as it is,
 * when the last tensor-core product on this workspace gave up a bounded
 * wait (each workspace keeps that status of its own last product, so
 * problems running at the same time never see each other's).  A NaN or Inf in A or B makes a whole row
 * (column) of C and the checksums covering it non-finite: each such element
 * is reported ABFT_KIND_NONFINITE_CORRECTED (recomputed, still non-finite),
 * its lines ABFT_KIND_UNCORRECTABLE, and the status is
 * ABFT_ERR_UNCORRECTABLE; the finite elements are left as they are. */
abft_status abft_verify_correct(const abft_desc* desc, void* C, void* ws, int32_t reread_C,
                                const int32_t* erased_blocks, int32_t n_erased, abft_fault* report,
                                int32_t max_reports, int32_t* n_reports, void* stream);

/* Erasure recovery (section 2.1: the lost part is the checksum minus the
 * surviving parts; section 3.3: the reduction step of a recovery).  Rebuilds
 * block (bi, bj) of the erasure grid as C_IJ = S_J - sum_{I' != I} C_I'J in
 * binary64, then re-checks the rebuilt block's column lines.  Call it after
 * abft_verify_correct (which must list the block as erased), because it reads
 * the rest of the block column.  report_entry (host, may be NULL) receives a
 * kind-4 entry.  SYNCHRONISES `stream`.  ABFT_ERR_UNCORRECTABLE when the
 * rebuilt block fails its checks. */
abft_status abft_recover_block(const abft_desc* desc, void* C, void* ws, int32_t bi, int32_t bj,
                               abft_fault* report_entry, void* stream);

/* Several erased blocks at once (section 2.1: with f block checksums, f lost
 * blocks of a block column follow from the checksums and the survivors).  The
 * grid carries grid_f block checksums S^(l) = sum_I c_{l,I} A_I (B), l < f, with
 * c_{l,I} = x_I^l, x_I = (2I+1-grid_p) / 2^e, 2^e > grid_p (distinct nodes: every
 * f x f minor is nonsingular; l = 0 is the plain sum).  blocks: host (bi, bj)
 * pairs, n_blocks <= 16, each listed once; a block column with t erased blocks
 * solves, for every element position, the t x t system of its first t
 * checksums in binary64 (the inverse is formed on the host), then the rebuilt
 * blocks' column lines are checked again.  report (host, n_blocks entries, may
 * be NULL) receives one kind-4 entry per block.  ABFT_ERR_UNCORRECTABLE, with
 * nothing launched, when a block column has more erased blocks than grid_f;
 * ABFT_ERR_UNCORRECTABLE also when a rebuilt block fails its checks.
 * SYNCHRONISES `stream`. */
abft_status abft_recover_blocks(const abft_desc* desc, void* C, void* ws, const int32_t* blocks,
                                int32_t n_blocks, abft_fault* report, void* stream);

/* Block rebuild when the block rows of one problem are spread over several
 * GPUs (section 3.1: the process grid holds the blocks; section 3.3: a lost
 * block is the block checksum minus the survivors, formed by one reduction
 * over the processes of its block column).  Each rank holds some block rows
 * of C as a problem of its own (desc with grid_p = its block rows, grid_q as
 * the global grid); one rank also holds the global block checksum rows
 * S = sum_I C_I of every block row in its workspace (its encoded S_A rows are
 * the reduction of every rank's local sum of A blocks before its product).
 *
 * abft_block_partial writes this rank's share of the rebuild of a block of
 * block column bj into out (device, bs x bc binary64, row-major, ld = bc;
 * bs = m / grid_p, bc = n / grid_q):
 *   out = (with_checksum ? S_bj : 0) - sum_{local block rows I != bi_skip} C_I,bj
 * (bi_skip = -1 when the lost block is not on this rank; with_checksum = 1 on
 * the rank that holds S, whose ws is then read).  Summing every rank's out
 * (one reduction, e.g. an NCCL reduce to the rank of the lost block) gives
 * the lost block.  ws may be NULL when with_checksum = 0.  Asynchronous.
 *
 * abft_block_restore writes sum (device, bs x bc binary64, as above) into
 * block (bi, bj) of C, rounded to C's type, and re-checks the block's column
 * lines against this workspace's element checksums.  report_entry (host, may
 * be NULL) receives a kind-4 entry.  ABFT_ERR_UNCORRECTABLE when the rebuilt
 * block fails its checks; ABFT_ERR_TIMEOUT (nothing written) when this
 * workspace's last tensor-core product timed out.  SYNCHRONISES `stream`.
 * Call abft_verify_correct (listing the block as erased) first on every rank,
 * since the shares read the rest of the block column. */
abft_status abft_block_partial(const abft_desc* desc, const void* C, const void* ws,
                               int32_t bi_skip, int32_t bj, int32_t with_checksum, double* out,
                               void* stream);
abft_status abft_block_restore(const abft_desc* desc, void* C, void* ws, int32_t bi, int32_t bj,
                               const double* sum, abft_fault* report_entry, void* stream);

/* Fault injection for tests and benchmarks (the paper's stress test kills
 * processes, section 4.3; here faults are bit flips and erasures chosen on the
 * host).  abft_inject_bitflips XORs bit bits[t] of element (rows[t], cols[t])
 * of C (host arrays of length count).  abft_erase_block fills block (bi, bj)
 * of the erasure grid with NaN.  Asynchronous. */
abft_status abft_inject_bitflips(const abft_desc* desc, void* C, const int64_t* rows,
                                 const int64_t* cols, const int32_t* bits, int32_t count,
                                 void* stream);
abft_status abft_erase_block(const abft_desc* desc, void* C, int32_t bi, int32_t bj, void* stream);

/* ---------------------------------------------------------------------------
 * Grouped products: many independent bf16 problems C_p = A_p B_p, each with
 * the encoded operands of Eq. (1) and the checks of section 2.2, executed by
 * one persistent product launch (and one encode / verify pass) for the whole
 * group.  The paper treats one distributed product; the grouping is a
 * batching layer over that method with no counterpart in the paper.
 *
 * Per problem: A (m x k, lda) and B (k x n, ldb) bf16 row-major on the device,
 * 16-byte aligned, lda and ldb multiples of 8; C (m x n, ldc) fp32.  Verify
 * blocks are 128 rows x 256 columns (weights 1..128 / 1..256 scaled by 2^-7 /
 * 2^-8, local to the block).  Product tiles are 128 rows x (64 * boxes_per_tile)
 * columns; a problem's checksum rows and columns are appended as 64-row halves
 * and 64-column boxes after its data, so they share the last data tiles.
 *
 * Ownership: the group object (host) holds the problem list, the tuning and a
 * captured CUDA graph; the caller's workspace (abft_group_workspace_bytes,
 * 256-byte aligned, bound with abft_group_bind) holds every device table and
 * per-problem checksum region.  The operand and result pointers given at
 * creation are used by every later call.  Calls are stream-ordered and
 * asynchronous unless marked SYNCHRONISES.
 * ------------------------------------------------------------------------- */
typedef struct {
  int64_t m, n, k;        /* C = A B; 1 <= m, n <= 2^20, 1 <= k <= 2^24    */
  int64_t lda, ldb, ldc;  /* leading dimensions in elements                */
  const void* A;          /* device, bf16                                  */
  const void* B;          /* device, bf16                                  */
  void* C;                /* device, fp32                                  */
} abft_problem;

typedef struct abft_group_s* abft_group;

typedef struct {
  int32_t boxes_per_tile; /* 4: 128 x 256 tiles; 2: 128 x 128 tiles          */
  int32_t order;          /* 0: problems in the given order; 1: by decreasing k */
} abft_group_tuning;

/* Where problem p's checksum results live in the workspace (byte offsets,
 * 256-byte aligned).  acs: R16 x acs_ld bf16 rows (per verify block I: rows 4I,
 * 4I+1 = hi, lo pieces of e^T A_I; 4I+2, 4I+3 = of w^T A_I); bcs: k x bcs_ld bf16,
 * the same 4 columns per verify column block; E16: R16 x n fp32 products of the
 * acs rows with B; F16: m x C16 fp32 products of A with the bcs columns (the
 * expected checksum of a line is the sum of its hi and lo products); nArow (m),
 * nAblk (4 nvr), nBcol (n), nBblk (4 nvc): binary64 norms of the thresholds,
 * as in abft_ws_layout. */
typedef struct {
  size_t acs, bcs, E16, F16, obs_col, obs_row, nArow, nAblk, nBcol, nBblk;
  int64_t nvr, nvc, R16, C16, acs_ld, bcs_ld;
} abft_group_layout;

/* Validates the problems (ABFT_ERR_INVALID with nothing created on a bad
 * one; dtype must be ABFT_BF16) and lays out the workspace.  tau_safety as in
 * abft_desc.  Host only. */
abft_status abft_group_create(const abft_problem* problems, int32_t count, int32_t dtype,
                              double tau_safety, abft_group* out);
size_t abft_group_workspace_bytes(abft_group g);
abft_status abft_group_problem_layout(abft_group g, int32_t p, abft_group_layout* out);
/* Builds the device tables (problem records, tensor maps, tile lists) in ws.
 * SYNCHRONISES `stream`. */
abft_status abft_group_bind(abft_group g, void* ws, size_t ws_bytes, void* stream);
/* Schedule tuning: tile width and problem order (default {4, 1}).  Rebuilds
 * the tables (SYNCHRONISES) and drops a captured graph. */
abft_status abft_group_set_tuning(abft_group g, const abft_group_tuning* t, void* stream);
abft_status abft_group_get_tuning(abft_group g, abft_group_tuning* t);
/* Autotuner: times `reps` checksum products of every tuning candidate and
 * keeps the fastest (*chosen, *best_ms; best_ms = -1 when the choice came from
 * the cache).  With the environment variable ABFT_TUNE_CACHE naming a file, a
 * group of the same shapes reuses the recorded choice and new choices are
 * appended.  Runs the product, so it overwrites every C and the checksum
 * results: encode and multiply again afterwards.  SYNCHRONISES `stream`. */
abft_status abft_group_autotune(abft_group g, int32_t reps, abft_group_tuning* chosen,
                                double* best_ms, void* stream);
/* Encode every problem's operands (section 2.1, Eq. (1)): checksum rows of A
 * and checksum columns of B as bf16 hi + lo pieces, and the norms of the
 * detection thresholds. */
abft_status abft_group_encode(abft_group g, void* stream);
/* The product of every problem.  checksums = 1: the ABFT product (data,
 * checksum rows and columns, observed sums of every data tile, armed epilogue
 * faults); 0: the same kernel on the data tiles only. */
abft_status abft_group_gemm(abft_group g, int32_t checksums, void* stream);
/* Detect / locate / correct every problem from the observed sums (as
 * abft_verify_correct with reread_C = 0).  _enqueue is asynchronous and may be
 * captured; _report SYNCHRONISES and returns the entries sorted by (problem,
 * row, col, kind) with the status rules of abft_verify_correct;
 * _verify_correct is both. */
abft_status abft_group_verify_enqueue(abft_group g, void* stream);
abft_status abft_group_report(abft_group g, abft_fault* report, int32_t max_reports,
                              int32_t* n_reports, void* stream);
abft_status abft_group_verify_correct(abft_group g, abft_fault* report, int32_t max_reports,
                                      int32_t* n_reports, void* stream);
/* Arms `count` (<= 256) bit flips of accumulator outputs: bit bits[t] of
 * element (rows[t], cols[t]) of problem problem[t] flips in the epilogue of
 * every later checksum product, before the store and the observed sums
 * (count = 0 disarms).  Host arrays. */
abft_status abft_group_set_epilogue_faults(abft_group g, const int32_t* problem,
                                           const int64_t* rows, const int64_t* cols,
                                           const int32_t* bits, int32_t count, void* stream);
/* CUDA graph of one step: the product (checksums as in abft_group_gemm) and,
 * with checksums, the verify enqueue.  Captured on `stream` (not the legacy
 * default stream); abft_group_launch replays it. */
abft_status abft_group_capture(abft_group g, int32_t checksums, void* stream);
abft_status abft_group_launch(abft_group g, void* stream);
abft_status abft_group_destroy(abft_group g);

/* Number of CUDA kernels this library has launched in this process so far
 * (all threads, all devices).  Host-side counter; never synchronises. */
int64_t abft_kernel_launches(void);

/* Thread-local message describing the last non-OK status of this thread. */
const char* abft_last_error(void);

/* Library version (major * 100 + minor). */
int32_t abft_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ABFT_H */
