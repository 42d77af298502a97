/*
 * evp.h -- C ABI of libevp, a GB300 (sm_103a) implementation of the search
 * hot path of "Ultra-Quantisation: Efficient Embedding Search via 1.58-bit
 * Encodings" (Connor, Dearle, Claydon; arXiv 2506.00528).
 *
 * The path: float32 embeddings are mapped to their nearest {x,d}
 * Equi-Voronoi-Polytope vertex (a ternary vector with exactly x non-zeros,
 * Sec. 2.3-2.4) stored as two bitplanes (Sec. 5.1.2); a query batch is
 * compared exhaustively with a database of such codes using the integer
 * proxy distance Delta (notation table, Sec. 2.6); the k nearest are kept
 * per query; optionally a shortlist is re-ordered by the original float
 * vectors (Sec. 5.3).
 *
 * Conventions shared by every call:
 *  - Array arguments are DEVICE pointers owned by the caller unless stated
 *    otherwise.  The library keeps no pointer after a call returns (except
 *    inside an evp_db_t, which borrows its arrays until evp_db_destroy).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream: they enqueue kernels
 *    and return.
 *  - Argument errors are detected on the host, returned immediately, and
 *    nothing is launched.  Errors that depend on the data (non-finite
 *    inputs, out-of-range shortlist ids, a device wait that timed out) are
 *    written to *dev_status, a device int32 that the caller sets to 0
 *    beforehand and reads after synchronising the stream; the first error
 *    written wins.  dev_status may be NULL, in which case such errors are
 *    not reported.  Outputs are unspecified when any status is not EVP_OK.
 *  - All entry points are safe to call from several host threads on
 *    different streams; calls that share an output or workspace buffer
 *    must be ordered by the caller.
 *
 * Packed code layout (the boundary format).  W = ceil(d/64).  One code is
 * 2W uint64 words, row-major, one row per vector: words [0, W) hold the
 * v+ plane (bit set where the element is +1) and words [W, 2W) the v-
 * plane (bit set where the element is -1).  Dimension j is bit (j mod 64)
 * of word floor(j/64) of its plane.  Bits at j >= d are 0.  Database
 * arrays passed to ternary_knn must be 16-byte aligned.
 */
#ifndef EVP_H
#define EVP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EVP_OK = 0,
    EVP_ERR_INVALID = 1,     /* bad argument (host-detected)                  */
    EVP_ERR_NONFINITE = 2,   /* NaN or infinity in a float input              */
    EVP_ERR_NO_MEMORY = 3,   /* workspace too small / allocation refused      */
    EVP_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up            */
    EVP_ERR_CUDA = 5,        /* a CUDA runtime call failed                    */
    EVP_ERR_UNSUPPORTED = 6, /* valid request outside this build's limits     */
    EVP_ERR_RANGE = 7        /* an index argument lies outside its array      */
} evp_status_t;

/* Limits of this build. */
#define EVP_MAX_D_ENCODE 2048   /* evp_encode: d <= 2048                       */
#define EVP_MAX_D_SCAN   1024   /* ternary_knn: d <= 1024                      */
#define EVP_MAX_K        1024   /* ternary_knn: k <= 1024                      */
#define EVP_MAX_SHORTLIST 4096  /* rerank: n <= 4096                           */
#define EVP_MAX_D_RERANK 4096   /* rerank: d <= 4096                           */

/* Human-readable name of a status code (static string, never NULL). */
const char* evp_status_string(int32_t status);

/* Library version, major*10000 + minor*100 + patch. */
int32_t evp_version(void);

/* W = ceil(d/64): uint64 words per bitplane; a packed code has 2W words.
 * Returns 0 for d < 1. */
int32_t evp_words(int32_t d);

/* The x of Sec. 5.1.1: the smallest x in [1, d] maximising the vertex count
 * C(d,x) * 2^x, which is floor((2d+1)/3).  Returns 0 for d < 1. */
int32_t evp_default_x(int32_t d);

/* ---------------------------------------------------------------------
 * evp_encode -- nearest {x,d} EVP vertex of each row (Sec. 2.4).
 *
 * For each row u of U the x elements of largest |u_i| are kept, +1 where
 * u_i is not negative and -1 where u_i < 0, every other element 0
 * (Sec. 2.4, steps 1-3), and the result is packed as above.
 * Readings where the paper is silent: magnitudes compare by their IEEE-754
 * bits with the sign cleared; equal magnitudes are taken lowest index
 * first; a selected +0.0 or -0.0 becomes +1, so every code has exactly x
 * non-zeros.  The float bytes are used as given (rows are expected to be
 * l2-normalised, Sec. 1.1, but the code does not depend on the scale).
 *
 *   U          [n][d] float32, row-major, device.
 *   n          rows, n >= 0 (n == 0 is a no-op).
 *   d          1 <= d <= EVP_MAX_D_ENCODE.
 *   x          1 <= x <= d.
 *   T          [n][2W] uint64 output, device.
 *   dev_status receives EVP_ERR_NONFINITE if any U element is NaN or
 *              infinite (the affected codes are then unspecified).
 * Returns EVP_OK, EVP_ERR_INVALID (null pointer with n > 0, d or x out of
 * range), EVP_ERR_UNSUPPORTED (d > EVP_MAX_D_ENCODE) or EVP_ERR_CUDA.
 * ------------------------------------------------------------------- */
int32_t evp_encode(const float* U, int64_t n, int32_t d, int32_t x,
                   uint64_t* T, int32_t* dev_status, void* stream);

/* ---------------------------------------------------------------------
 * ternary_knn -- exhaustive k-nearest-neighbour scan in the proxy space.
 *
 * Delta(q, s) = ||q - s||^2 over the ternary vectors, which for two codes
 * with x non-zeros each is 2x - 2*b2sp(q, s), with b2sp the bitplane
 * scalar product of Sec. 5.1.2:
 *   b2sp = bsp(q+,s+) + bsp(q-,s-) - bsp(q+,s-) - bsp(q-,s+),
 *   bsp(a,b) = popcount(a AND b).
 * Delta is even and lies in [0, 4x]; smaller is nearer.  For each query
 * the k database rows with the smallest (Delta, row index) pairs are
 * returned in ascending order: equal Delta is broken by the lower row
 * index, so the result is unique (the exhaustive search of Sec. 5.3 and of
 * the 100-query scans of Table 5).
 *
 *   Q          [nq][2W] packed query codes, device.
 *   nq         queries, nq >= 0 (0 is a no-op).
 *   S          [ns][2W] packed database codes, device, 16-byte aligned.
 *   ns         1 <= ns < 2^31 rows.
 *   d          1 <= d <= EVP_MAX_D_SCAN.
 *   x          non-zeros per code, 1 <= x <= d (the same x for Q and S).
 *   k          1 <= k <= min(ns, EVP_MAX_K).
 *   ids        [nq][k] int64 output: database row indices.
 *   dist       [nq][k] int32 output: Delta of each returned row.
 *   ws         device workspace of at least ternary_knn_workspace(...)
 *              bytes, 256-byte aligned; its contents on entry are ignored.
 *              The size returned for nq queries also serves every call
 *              with fewer queries and the same other arguments.
 *   ws_bytes   size of ws.
 * Returns EVP_OK, EVP_ERR_INVALID, EVP_ERR_NO_MEMORY (ws_bytes too small),
 * EVP_ERR_UNSUPPORTED (d > EVP_MAX_D_SCAN or k > EVP_MAX_K) or
 * EVP_ERR_CUDA.  dev_status may receive EVP_ERR_TIMEOUT.
 * ------------------------------------------------------------------- */
size_t ternary_knn_workspace(int64_t nq, int64_t ns, int32_t d, int32_t k);

int32_t ternary_knn(const uint64_t* Q, int64_t nq, const uint64_t* S, int64_t ns,
                    int32_t d, int32_t x, int32_t k, int64_t* ids, int32_t* dist,
                    void* ws, size_t ws_bytes, int32_t* dev_status, void* stream);

/* ---------------------------------------------------------------------
 * Single-operand translation (Sec. 6): the database is mapped to EVP
 * vertices, the query keeps its values.  Here the query is held as int8, so
 * that every score is an exact integer and results are reproducible bit for
 * bit (the paper fixes no precision for the untranslated operand; int8
 * keeps the recall of float queries on this build's synthetic data).
 *
 * evp_quantize_i8: per-query symmetric int8.  m = max_i |q_i|, scale =
 * 127 / m in float32, q8_i = q_i * scale rounded to the nearest integer,
 * ties to even (IEEE float32 arithmetic throughout); m = 0 gives zeros.
 *   Q      [nq][d] float32, device.     Q8  [nq][d] int8 output, device.
 *   dev_status receives EVP_ERR_NONFINITE for a NaN or infinite element
 *   (that row is then all zero).
 * Returns EVP_OK, EVP_ERR_INVALID or EVP_ERR_CUDA.
 *
 * ternary_knn_i8q: exhaustive search of Sec. 5.3 with the masked-addition
 * score of Sec. 5.1.2 -- score(q, s) = sum of q8_i where s_i = +1 minus
 * the sum where s_i = -1 (= <q8, s>, no multiplication needed) -- the k
 * rows with the largest score per query, equal scores by lower row index.
 *   Q8     [nq][d] int8 queries, device.
 *   S      [ns][2W] packed database codes (as for ternary_knn), 16-byte
 *          aligned; every code has x non-zeros.
 *   ids    [nq][k] int64 output; score [nq][k] int32 output (descending).
 *   ws     workspace of ternary_knn_i8q_workspace(...) bytes (0 means the
 *          shape is not supported), 256-byte aligned.
 * Runs on the tensor cores: database tiles unpacked on chip (as
 * EVP_PATH_MMA_PACKED) against each query split exactly as 16 hi + lo with
 * e4m3 parts, passes of up to 32 queries.  Limits as EVP_PATH_MMA_PACKED:
 * d <= 768 with ceil(d/64) even, k <= 256 (else EVP_ERR_UNSUPPORTED).
 * Returns EVP_OK, EVP_ERR_INVALID, EVP_ERR_UNSUPPORTED, EVP_ERR_NO_MEMORY
 * or EVP_ERR_CUDA; dev_status may receive EVP_ERR_TIMEOUT.
 * ------------------------------------------------------------------- */
int32_t evp_quantize_i8(const float* Q, int64_t nq, int32_t d, int8_t* Q8, int32_t* dev_status,
                        void* stream);
size_t ternary_knn_i8q_workspace(int64_t nq, int64_t ns, int32_t d, int32_t k);
int32_t ternary_knn_i8q(const int8_t* Q8, int64_t nq, const uint64_t* S, int64_t ns, int32_t d,
                        int32_t x, int32_t k, int64_t* ids, int32_t* score, void* ws,
                        size_t ws_bytes, int32_t* dev_status, void* stream);

/* ---------------------------------------------------------------------
 * Sparse codes for small x (Sec. 6, "different EVPs": fewer non-zeros are
 * less accurate but faster).  A sparse code lists the x non-zero
 * dimensions of a vertex in ascending order, one uint16 each: bits 0-14 the
 * dimension, bit 15 set where the element is -1; [n][x] row-major.  At
 * x = 64, d = 768 it is 128 bytes per row against 192 for the bitplanes.
 *
 * evp_pack_sparse: packed bitplane codes T [n][2W] -> E [n][x] (device).
 * A row with other than x non-zeros gets EVP_ERR_RANGE in dev_status (its
 * first min(count, x) entries are written, the rest 0).  Returns EVP_OK,
 * EVP_ERR_INVALID (d > 32768 among others) or EVP_ERR_CUDA.
 *
 * ternary_knn_sparse: exhaustive kNN (Sec. 5.3) of packed ternary queries Q
 * [nq][2W] over a sparse database E [ns][x] (16-byte aligned): for each
 * query the k rows with the smallest (Delta, row), Delta = ||q - s||^2 --
 * the same results as ternary_knn over the bitplane form of the same codes.
 * Delta is computed by masked addition (Sec. 5.1.2): per database row, one
 * table lookup per non-zero.  Queries are scanned in passes of 4.  Needs
 * 8 <= x <= 120 with x a multiple of 8, d <= 1024 and k <= 256 (else
 * EVP_ERR_UNSUPPORTED; ternary_knn_sparse_workspace then returns 0).
 * Workspace: ternary_knn_sparse_workspace(...) bytes, 256-byte aligned.
 * Returns EVP_OK, EVP_ERR_INVALID, EVP_ERR_UNSUPPORTED, EVP_ERR_NO_MEMORY or
 * EVP_ERR_CUDA.
 * ------------------------------------------------------------------- */
int32_t evp_pack_sparse(const uint64_t* T, int64_t n, int32_t d, int32_t x, uint16_t* E,
                        int32_t* dev_status, void* stream);
size_t ternary_knn_sparse_workspace(int64_t nq, int64_t ns, int32_t d, int32_t x, int32_t k);
int32_t ternary_knn_sparse(const uint64_t* Q, int64_t nq, const uint16_t* E, int64_t ns,
                           int32_t d, int32_t x, int32_t k, int64_t* ids, int32_t* dist, void* ws,
                           size_t ws_bytes, int32_t* dev_status, void* stream);

/* ---------------------------------------------------------------------
 * ternary_knn_static -- ternary_knn (popcount path) that allocates
 * nothing.  The paper has no counterpart; this exists for callers that
 * cannot allocate device memory: serving threads that must never enter the
 * device allocator (an allocation can wait on device-wide
 * synchronisation and so stall a latency-bound loop), plugins handed raw
 * device pointers by a host framework that owns all allocation, and plain
 * C callers with no allocator of their own.  Inputs and outputs are the
 * caller's, as in ternary_knn; the workspace is a fixed
 * EVP_STATIC_SCRATCH_BYTES (16 MiB) array inside the library, present on
 * every GPU that loads it until the process exits.  A request whose
 * popcount-path workspace (ternary_knn_path_workspace(nq, ns, d, k,
 * EVP_PATH_POPC)) exceeds that size is rejected with EVP_ERR_NO_MEMORY
 * before anything is launched.  The first call on each device looks up the
 * array's device address (with that device current) and caches it, so make
 * that first call before any stream capture; a device reset
 * (cudaDeviceReset) reloads the library's device code and invalidates the
 * cached address, so the entry point must not be used after one.  All
 * calls share the one array and it keeps the previous call's contents (each
 * call re-initialises what it reads): calls that overlap on the GPU race on
 * it, so the caller must order them (one stream, or events).  Results are
 * identical to ternary_knn with EVP_PATH_POPC.
 * ------------------------------------------------------------------- */
#define EVP_STATIC_SCRATCH_BYTES (16u << 20)
int32_t ternary_knn_static(const uint64_t* Q, int64_t nq, const uint64_t* S, int64_t ns,
                           int32_t d, int32_t x, int32_t k, int64_t* ids, int32_t* dist,
                           int32_t* dev_status, void* stream);

/* Scan paths.  All return identical results.
 *   EVP_PATH_POPC  bitplane popcount scan on the integer pipe: reads the
 *                  packed codes once per 16 queries; best for up to three
 *                  queries.
 *   EVP_PATH_MMA   tensor-core scan (tcgen05 kind::mxf4: 4-bit e2m1 operands
 *                  holding -1/0/+1, unit block scales, float32
 *                  accumulation, exact) with the queries as the 128-row
 *                  side: the codes are expanded to half a byte per element
 *                  (in the workspace when S is given packed, or once for a
 *                  database created with EVP_DB_TENSOR_COPY).
 *                  Each database slice keeps kl keys per query: kl < k (a
 *                  power of two, 16-128) when the slices are many enough,
 *                  with a check of every list's tail after the merge and a
 *                  rescan of the rare slice that may have held more (the
 *                  result stays exact); otherwise kl = k, and for k > 128
 *                  a 128-query tile then serves fewer queries (64, 32, 16).
 *                  Best for large batches.
 *   EVP_PATH_MMA_PACKED  tensor-core scan with the database as the 128-row
 *                  side: reads the packed codes once per 64 queries and
 *                  unpacks each tile on chip into tensor memory; needs
 *                  d <= 768 with ceil(d/64) even and k <= 256 (else
 *                  EVP_ERR_UNSUPPORTED) and at most 2^20 * 256 rows; best
 *                  for medium batches.
 *   EVP_PATH_AUTO  POPC for nq <= EVP_AUTO_POPC_MAX_NQ; MMA_PACKED (where
 *                  supported) up to EVP_AUTO_PACKED_MAX_NQ queries against a
 *                  resident database holding its e2m1 copy, and up to
 *                  EVP_AUTO_PACKED_MAX_NQ_NO_COPY otherwise (MMA would first
 *                  expand the database); MMA beyond.  Where the packed path
 *                  does not apply: MMA when nq > 16 (> 8 with a resident
 *                  copy), POPC otherwise.  This is what ternary_knn and
 *                  evp_db_knn/evp_db_search use.
 * The tensor-core paths assume every code has exactly x non-zeros (as
 * evp_encode produces): they compute Delta as 2x - 2*b2sp.  The POPC path
 * computes ||q - s||^2 directly. */
#define EVP_PATH_AUTO 0
#define EVP_PATH_POPC 1
#define EVP_PATH_MMA  2
#define EVP_PATH_MMA_PACKED 3
#define EVP_AUTO_POPC_MAX_NQ 2
#define EVP_AUTO_PACKED_MAX_NQ 32
#define EVP_AUTO_PACKED_MAX_NQ_NO_COPY 128
#define EVP_MMA_MAX_K 1024

size_t ternary_knn_path_workspace(int64_t nq, int64_t ns, int32_t d, int32_t k,
                                  int32_t path);

int32_t ternary_knn_path(const uint64_t* Q, int64_t nq, const uint64_t* S, int64_t ns,
                         int32_t d, int32_t x, int32_t k, int64_t* ids, int32_t* dist,
                         void* ws, size_t ws_bytes, int32_t* dev_status, void* stream,
                         int32_t path);

/* ---------------------------------------------------------------------
 * evp_merge_topk -- merge per-shard kNN results into the global top-k.
 *
 * For a database split into row shards (e.g. one per GPU, Sec. 5.3's
 * exhaustive search run on each part), ids [nlists][nq][k] (int64,
 * global row ids in [0, 2^31)) and dist [nlists][nq][k] (int32 Delta), each
 * list sorted by (Delta, id) as ternary_knn returns them, are merged per
 * query into the k smallest (Delta, id) pairs.  A list may end early with
 * id -1 (a shard with fewer than k rows).  The result equals ternary_knn
 * over the whole database when every shard returned its own k nearest.
 * Workspace: evp_merge_topk_workspace(...) bytes, 256-byte aligned.
 * Returns EVP_OK, EVP_ERR_INVALID, EVP_ERR_UNSUPPORTED (k > EVP_MAX_K or
 * nlists > 1024), EVP_ERR_NO_MEMORY or EVP_ERR_CUDA; dev_status receives
 * EVP_ERR_RANGE for an id >= 2^31.
 * ------------------------------------------------------------------- */
size_t evp_merge_topk_workspace(int64_t nq, int32_t nlists, int32_t k);
int32_t evp_merge_topk(const int64_t* ids, const int32_t* dist, int64_t nq, int32_t nlists,
                       int32_t k, int64_t* out_ids, int32_t* out_dist, void* ws, size_t ws_bytes,
                       int32_t* dev_status, void* stream);

/* ---------------------------------------------------------------------
 * rerank -- re-order a shortlist by the original vectors (Sec. 5.3: n > k
 * proxy results are re-ordered in the original space and the best k
 * kept).
 *
 * score(q, s) = <q, s> in float32 (for l2-normalised rows this orders as
 * cosine similarity and as Euclidean distance, Sec. 1.1), summed in a
 * fixed order: per lane of a warp a running FMA over a strided share of
 * the d elements, then a five-level butterfly over the 32 lanes.  Output
 * per query: the k best entries by (score descending, row index
 * ascending); -0.0 is treated as +0.0.
 *
 *   Q          [nq][d] float32 queries, device.
 *   S          [ns][d] float32 database rows, device.
 *   shortlist  [nq][n] int64 row ids; -1 marks an empty entry (skipped).
 *   n          1 <= n <= EVP_MAX_SHORTLIST.
 *   k          1 <= k <= n.
 *   ids        [nq][k] int64 output; positions beyond the number of
 *              non-empty entries get -1.
 *   scores     [nq][k] float32 output; -infinity where ids is -1.
 * dev_status receives EVP_ERR_RANGE for an id outside [-1, ns) (the entry
 * is then skipped) and EVP_ERR_NONFINITE for a non-finite score.
 * Returns EVP_OK, EVP_ERR_INVALID, EVP_ERR_UNSUPPORTED (d or n above the
 * limits) or EVP_ERR_CUDA.
 * ------------------------------------------------------------------- */
int32_t rerank(const float* Q, int64_t nq, const float* S, int64_t ns, int32_t d,
               const int64_t* shortlist, int32_t n, int32_t k,
               int64_t* ids, float* scores, int32_t* dev_status, void* stream);

/* ---------------------------------------------------------------------
 * Resident database (the serving form of the path: a database encoded
 * once, Sec. 1.1's "pre-processing of S before q becomes available", and
 * searched by many query batches).
 *
 * evp_db_create borrows T ([ns][2W] packed codes, device, 16-byte aligned)
 * and U ([ns][d] float32 rows, device, or NULL if no rerank is wanted); the
 * caller keeps both alive and unchanged until evp_db_destroy.  With
 * EVP_DB_TENSOR_COPY the handle also owns a half-byte-per-element e2m1 copy
 * of the codes ([ns][Kp] bytes, Kp = d/2 rounded up to 128; allocated with
 * cudaMalloc, filled on `stream`, which is synchronised before returning)
 * so that the tensor-core scan need not rebuild it per call.
 * Returns EVP_OK, EVP_ERR_INVALID, EVP_ERR_UNSUPPORTED (d > EVP_MAX_D_SCAN),
 * EVP_ERR_NO_MEMORY (the copy could not be allocated) or EVP_ERR_CUDA.
 *
 * evp_db_knn: ternary_knn_path against the resident database (same
 * arguments, same results).
 *
 * evp_db_search: the whole path for float32 queries Q [nq][d] (device):
 * evp_encode -> scan for the n_shortlist nearest by Delta -> rerank of
 * that shortlist by <q, s> over U -> ids [nq][k] (int64) and scores
 * [nq][k] (float32), k <= n_shortlist <= min(ns, EVP_MAX_K).  Needs U.
 * The scan path is chosen as by ternary_knn.
 *
 * evp_db_search_host: the same with HOST buffers: Q_host is copied to the
 * device, results are copied back, all asynchronously on `stream`; the host
 * buffers must stay valid until the stream has passed the call (pinned
 * memory makes the copies truly asynchronous).
 *
 * Workspaces are caller-owned device memory (256-byte aligned) of at least
 * the size the matching *_workspace call returns; the size for nq queries
 * also serves every call with fewer queries and the same other arguments.
 * ------------------------------------------------------------------- */
typedef struct evp_db* evp_db_t;
#define EVP_DB_TENSOR_COPY 1

int32_t evp_db_create(const uint64_t* T, const float* U, int64_t ns, int32_t d, int32_t x,
                      int32_t flags, void* stream, evp_db_t* out);
int32_t evp_db_destroy(evp_db_t db);
int32_t evp_db_dim(evp_db_t db);   /* d of the database (0 for NULL) */
int64_t evp_db_rows(evp_db_t db);  /* ns of the database (0 for NULL) */
const uint64_t* evp_db_codes(evp_db_t db);  /* the borrowed packed codes T */
size_t evp_db_knn_workspace(evp_db_t db, int64_t nq, int32_t k, int32_t path);
int32_t evp_db_knn(evp_db_t db, const uint64_t* Q, int64_t nq, int32_t k, int64_t* ids,
                   int32_t* dist, void* ws, size_t ws_bytes, int32_t* dev_status, void* stream,
                   int32_t path);
size_t evp_db_search_workspace(evp_db_t db, int64_t nq, int32_t n_shortlist, int32_t k);
int32_t evp_db_search(evp_db_t db, const float* Q, int64_t nq, int32_t n_shortlist, int32_t k,
                      int64_t* ids, float* scores, void* ws, size_t ws_bytes,
                      int32_t* dev_status, void* stream);
/* evp_db_search with the scan path forced (EVP_PATH_*); same results. */
size_t evp_db_search_path_workspace(evp_db_t db, int64_t nq, int32_t n_shortlist, int32_t k,
                                    int32_t path);
int32_t evp_db_search_path(evp_db_t db, const float* Q, int64_t nq, int32_t n_shortlist,
                           int32_t k, int64_t* ids, float* scores, void* ws, size_t ws_bytes,
                           int32_t* dev_status, void* stream, int32_t path);
size_t evp_db_search_host_workspace(evp_db_t db, int64_t nq, int32_t n_shortlist, int32_t k);
int32_t evp_db_search_host(evp_db_t db, const float* Q_host, int64_t nq, int32_t n_shortlist,
                           int32_t k, int64_t* ids_host, float* scores_host, void* ws,
                           size_t ws_bytes, int32_t* dev_status, void* stream);

/* ---------------------------------------------------------------------
 * Batched form: many query batches of uneven sizes against several
 * resident databases, planned once and replayed (no counterpart in the
 * paper; it batches the Sec. 5.3 search).
 *
 * An evp_batch_desc is either a whole-path search (Q = float32 queries
 * [nq][d] on the device, n_shortlist >= k, outputs ids and scores, as
 * evp_db_search) or a plain kNN (Q = NULL, Qc = packed codes [nq][2W],
 * outputs ids and dist, as evp_db_knn).  All pointers are device pointers
 * owned by the caller and must stay valid while the plan exists.
 *
 * evp_autotune times the popcount and both tensor-core scans (where they
 * apply) on a database for a query count (rounded up to a power of two)
 * and k, using the database's own rows as trial queries, and keeps the
 * fastest path per (GPU model, d, x, query-count bucket, k, row-count
 * bucket); *path_out receives it, *popc_ms (optional) the popcount time
 * and *mma_ms (optional) the faster tensor-core time; asking for a timing
 * forces a fresh measurement.  It allocates temporary device memory.
 * evp_autotune_save / evp_autotune_load write and read the tuner's
 * decisions (paths and fused tile shapes) as a text file, one "key value"
 * line each, so that a deployment tunes once per GPU model; loading merges
 * into the current table.  evp_autotune_clear empties it.
 *
 * evp_batch_plan_create checks every descriptor, picks each batch's path
 * with evp_autotune (EVP_BATCH_NO_TUNE: the automatic rule instead) and
 * allocates one workspace region per batch (the plan owns it).  Every batch
 * whose path is the fp4 tensor-core scan (EVP_PATH_MMA) and whose database
 * holds its tensor copy (EVP_DB_TENSOR_COPY) joins the fused scan (at most
 * 64 batches): one persistent launch over the work items -- (batch, query
 * unit, database slice) -- of all of them, after one launch that prepares
 * all their queries and before one final merge of all their queries.  The
 * fused scan's tile shape (database tiles per work item, scaled by each
 * batch's d so that items cost about the same) is timed on the plan's own
 * batches among a few candidates and remembered by the tuner
 * (EVP_BATCH_NO_TUNE: a fixed shape).  EVP_BATCH_SEPARATE runs every batch
 * with its own calls instead.
 * evp_batch_run enqueues all batches on `stream`: the fused scan there, the
 * other batches dealt over four forked streams that join back into
 * `stream`; with EVP_BATCH_GRAPH the first run captures this into a CUDA
 * graph (`stream` must not be the legacy default stream) and every run
 * launches the graph.  Results equal the per-batch evp_db_search /
 * evp_db_knn calls.  dev_status is shared by all batches (and baked into the
 * graph at capture).  evp_batch_plan_fused returns how many batches the
 * fused scan takes, evp_batch_plan_tile the tile shape of batch i (0 when
 * it is not fused).
 * ------------------------------------------------------------------- */
typedef struct {
    evp_db_t db;
    const float* Q;       /* float32 queries [nq][d], or NULL for a plain kNN */
    const uint64_t* Qc;   /* packed query codes [nq][2W] (plain kNN)          */
    int64_t nq;
    int32_t n_shortlist;  /* search: shortlist length by Delta (>= k)         */
    int32_t k;
    int64_t* ids;         /* [nq][k]                                          */
    float* scores;        /* search: [nq][k]                                  */
    int32_t* dist;        /* plain kNN: [nq][k] Delta                         */
} evp_batch_desc;
typedef struct evp_batch_plan* evp_batch_plan_t;
#define EVP_BATCH_GRAPH    1
#define EVP_BATCH_NO_TUNE  2
#define EVP_BATCH_SEPARATE 4

int32_t evp_autotune(evp_db_t db, int64_t nq, int32_t k, int32_t* path_out, float* popc_ms,
                     float* mma_ms, void* stream);
int32_t evp_autotune_clear(void);
int32_t evp_autotune_save(const char* path);
int32_t evp_autotune_load(const char* path);
int32_t evp_batch_plan_create(const evp_batch_desc* batches, int32_t nb, int32_t flags,
                              void* stream, evp_batch_plan_t* out);
int32_t evp_batch_plan_path(evp_batch_plan_t plan, int32_t i);   /* chosen path of batch i */
int32_t evp_batch_plan_fused(evp_batch_plan_t plan);
int32_t evp_batch_plan_tile(evp_batch_plan_t plan, int32_t i);
size_t evp_batch_plan_workspace(evp_batch_plan_t plan);
int32_t evp_batch_run(evp_batch_plan_t plan, int32_t* dev_status, void* stream);
int32_t evp_batch_plan_destroy(evp_batch_plan_t plan);

/* ---------------------------------------------------------------------
 * Serving: a continuous-batching request loop over a resident database
 * (the served form of the Sec. 5.3 search; the paper has no serving
 * system).
 *
 * evp_server_create starts a host worker thread.  Each request (host
 * float32 queries Q_host [nq][d], k) is searched exactly as
 * evp_db_search_host would search it alone, with a shortlist of
 * min(shortlist_factor * k, EVP_MAX_K) rows by Delta reranked to k: the
 * worker coalesces pending requests with the same k, in arrival order, into
 * batches of at most max_batch_queries queries and runs up to `slots`
 * batches concurrently, each on its own stream with its own pinned staging
 * and device workspace.  Requests arriving while batches run are admitted
 * as soon as a slot frees up.  Results are bit-identical whether a request
 * runs alone or among others.
 *
 * Admission by memory: slots = min(max_slots, mem_budget_bytes / bytes of
 * one slot's workspace) (mem_budget_bytes <= 0 means one slot);
 * evp_server_create returns EVP_ERR_NO_MEMORY when not even one slot fits,
 * and evp_server_submit returns EVP_ERR_NO_MEMORY for a request larger than
 * a slot.
 *
 * evp_server_submit copies nothing at submission: Q_host, ids_host
 * ([nq][k] int64) and scores_host ([nq][k] float32) must stay valid until
 * evp_server_wait has returned EVP_OK for the request.  evp_server_wait
 * blocks up to timeout_us microseconds (EVP_ERR_TIMEOUT if the request is
 * not finished; it can be waited for again) and then releases the request;
 * *request_status is the device status of the request's batch and
 * *latency_us the time from submission to completion.  evp_server_stats
 * reports completed requests, queries, batches, pending requests and the
 * p50 / p99 / max latency of the requests completed since the last
 * evp_server_reset_stats.  evp_server_destroy finishes queued requests
 * (resuming a paused server) and joins the worker.
 * ------------------------------------------------------------------- */
typedef struct evp_server* evp_server_t;
typedef struct {
    int32_t device;             /* CUDA device holding the database            */
    int32_t max_batch_queries;  /* capacity of one batch (slot), in queries    */
    int32_t max_k;              /* largest k a request may ask for             */
    int32_t shortlist_factor;   /* shortlist length = factor * k (capped)      */
    int32_t max_slots;          /* batches in flight at most                   */
    int64_t mem_budget_bytes;   /* device bytes available for slot workspaces  */
} evp_server_config;
typedef struct {
    int64_t requests, queries, batches, pending;
    double p50_us, p99_us, max_us;
} evp_server_stats_t;

int32_t evp_server_create(evp_db_t db, const evp_server_config* cfg, evp_server_t* out);
int32_t evp_server_slots(evp_server_t s);
int32_t evp_server_submit(evp_server_t s, const float* Q_host, int64_t nq, int32_t k,
                          int64_t* ids_host, float* scores_host, int64_t* request_id);
int32_t evp_server_wait(evp_server_t s, int64_t request_id, int64_t timeout_us,
                        int32_t* request_status, double* latency_us);
int32_t evp_server_stats(evp_server_t s, evp_server_stats_t* out);
int32_t evp_server_reset_stats(evp_server_t s);
/* Stop (1) or resume (0) admitting new batches; batches in flight finish.
 * Requests keep queueing while paused.  Used to drain, and by tests to
 * stall the worker on the host. */
int32_t evp_server_pause(evp_server_t s, int32_t paused);
int32_t evp_server_destroy(evp_server_t s);

/* ---------------------------------------------------------------------
 * Kernel timing (measurement support; the paper has no counterpart).
 *
 * evp_timing_enable(1) makes every later call record a pair of CUDA events
 * on its stream around each launch of the library's kernels; (0) stops
 * recording.  evp_timing_read synchronises on the recorded events and
 * returns, for the kernel family `name` ("encode", "scan_init",
 * "scan_popc", "unpack_fp8", "scan_mma", "scan_mma_packed", "scan_i8q", "quantize",
 * "scan_sparse", "pack_sparse", "final_merge", "pack_lists", "rerank"), the number
 * of launches and their total
 * duration in milliseconds since the last evp_timing_reset.  Returns
 * EVP_OK, EVP_ERR_INVALID (null outputs) or EVP_ERR_CUDA.  Enabling adds
 * two event records per launch; leave it off outside measurements.
 * ------------------------------------------------------------------- */
int32_t evp_timing_enable(int32_t on);
int32_t evp_timing_reset(void);
int32_t evp_timing_read(const char* name, int64_t* launches, double* total_ms);

/* ---------------------------------------------------------------------
 * evp_probe_tensor_rate -- measured dense tensor-core rate (measurement
 * support for the roofline of the tensor-core scans; the paper has no
 * counterpart).
 *
 * Every SM (kind 0: tcgen05.mma.kind::f8f6f4 with e4m3 operands, K = 32;
 * kind 1: kind::f16 with bf16 operands, K = 16; kind 2: kind::mxf4 with
 * packed e2m1 operands and unit ue8m0 block scales, K = 64, the ternary
 * scan's form; float32 accumulation)
 * issues `iters` instructions of shape M x n x K back to back from one
 * thread, on operands resident in shared memory that hold +1, -1 and 0 in
 * equal shares (the values the scans contract).  cta_pair = 0: one CTA per
 * SM, M = 128; cta_pair = 1: CTA pairs (cta_group::2), M = 256.  n is a
 * multiple of 16 in [16, 256]; 1 <= iters <= 2^26.  kind | 0x100 fills
 * the operands with zeros instead, kind | 0x200 (e4m3 only) with random
 * finite bytes, to show whether the rate depends on the values.
 * kind | 0x400 (e4m3, n <= 128) takes the A operand from
 * tensor memory, as the packed scan does; kind | 0x800 (cta_pair = 0)
 * issues M = 64 instructions.  kind | 0x1000 (e4m3, A in shared memory)
 * adds a tcgen05.commit after every four instructions, kind | 0x2000 a
 * test of a completed mbarrier and a tcgen05 fence: the per-stage work of
 * a pipelined scan's issuing thread; kind | 0x3000 takes every four
 * instructions' operands from the next of four distinct buffers, as a scan
 * streaming fresh stages does; kind | 0x4000 switches between two
 * accumulators every 24 instructions (a scan's tile change); kind | 0x5000
 * has the other warps read tensor memory throughout (an epilogue);
 * kind | 0x6000 switches without restarting (accumulate = 1), kind | 0x7000
 * restarts (accumulate = 0) every 24 instructions without switching.
 * Synchronous: the launch
 * is timed with CUDA events on `stream`.  Outputs: *tflops =
 * 2 M n K iters x instruction issuers / elapsed time; *cycles_per_mma =
 * SM clocks per instruction on the issuing thread (averaged over SMs);
 * *ms = elapsed time.  (The int8 kind, kind::i8, does not exist on sm_103a:
 * ptxas rejects it for this target.)  Returns EVP_OK, EVP_ERR_INVALID,
 * EVP_ERR_NO_MEMORY (two small device buffers), EVP_ERR_TIMEOUT or
 * EVP_ERR_CUDA.
 * ------------------------------------------------------------------- */
int32_t evp_probe_tensor_rate(int32_t kind, int32_t cta_pair, int32_t n, int64_t iters,
                              double* tflops, double* cycles_per_mma, double* ms, void* stream);

/* ---------------------------------------------------------------------
 * Testing support for failure detection (the paper has no counterpart).
 *
 * evp_test_stall_producer(path, fills) arms a one-shot stall for the next
 * launch of the tensor-core scan `path` (EVP_PATH_MMA or
 * EVP_PATH_MMA_PACKED): the first CTA's copy producer stops after `fills`
 * stage fills, as a copy engine that never delivers would.  The scan's
 * bounded device waits (2 s) then expire: the call writes EVP_ERR_TIMEOUT
 * to dev_status, every CTA waits (bounded) for the copies and tensor-core
 * operations it issued, frees its tensor memory and exits, the outputs
 * are unspecified, and the device stays usable for later calls.  Nothing
 * faults.  fills < 0 disarms.  Returns EVP_OK, or EVP_ERR_INVALID for
 * another path.
 * ------------------------------------------------------------------- */
int32_t evp_test_stall_producer(int32_t path, int32_t fills);

#ifdef __cplusplus
}
#endif

#endif /* EVP_H */
