/*
 * oracle.h -- plain CPU oracle for the PolyMinHash signature path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA library: no headers, helpers, tables or constants.
 *
 * Every routine is the plain definition (or the paper's algorithm in the
 * paper's order) written out for readability, not speed.  Floating point is
 * fp64 (long double where stated); integer work is exact int64/int128.
 *
 * Polygon layout (shared with the callers, not with the CUDA library):
 *   xy      int32 [V][2]  interleaved vertex coordinates (x, y)
 *   offsets int64 [N+1]   polygon p owns vertices offsets[p] .. offsets[p+1]-1
 *   edges are (v_i, v_{(i+1) mod n}); the closing vertex is not repeated.
 */
#ifndef PMH_ORACLE_H
#define PMH_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- random point streams (reading of Sec. 3.2 "fixed seeds") ---- */
uint64_t orc_mix64(uint64_t z);
uint64_t orc_stream_seed(uint64_t seed, uint64_t k);
uint64_t orc_stream_value(uint64_t seed, uint64_t k, uint64_t i);
void orc_stream_points(uint64_t seed, uint64_t k, uint64_t i0, int64_t count,
                       uint32_t* x, uint32_t* y);

/* ---- lattice membership (reading of the "precise PnP" test, Sec. 3.2) ---- */
int orc_inside(const int32_t* xy, int64_t n, int64_t px, int64_t py);
int64_t orc_lattice_count(const int32_t* xy, int64_t n);
int orc_lattice_pair(const int32_t* a, int64_t na, const int32_t* b, int64_t nb,
                     int64_t* count_a, int64_t* count_b, int64_t* count_ab);
int64_t orc_area2(const int32_t* xy, int64_t n);
void orc_bbox(const int32_t* xy, int64_t n, int32_t* bbox4);

/* ---- Definition 2 / Algorithm 1 ---- */
int orc_sign(const int32_t* xy, const int64_t* offsets, int64_t n_polys,
             uint64_t seed, uint32_t K, uint32_t T, uint32_t* hashes,
             int nthreads);
int orc_sign_work(const int32_t* xy, const int64_t* offsets, int64_t n_polys,
                  uint64_t seed, uint32_t K, uint32_t T, uint32_t* hashes,
                  int64_t* points, int64_t* bbox_hits, int64_t* edge_tests);

/* ---- banding / hashmap buckets (Sec. 3.2 after Thm. 1, Sec. 5.2) ---- */
void orc_band_keys(const uint32_t* hashes, int64_t n, uint32_t K, uint32_t bands,
                   uint32_t rows, uint32_t T, uint64_t lsh_seed, uint64_t* keys);
int64_t orc_candidates(const uint32_t* qh, int64_t Q, const uint32_t* ph, int64_t N,
                       uint32_t K, uint32_t bands, uint32_t rows, uint32_t T,
                       int64_t* row_ptr, int32_t* cand, int64_t cap);

/* ---- Theorem 1 agreement estimate ---- */
void orc_agree(const uint32_t* qh, const uint32_t* ph, uint32_t K, uint32_t bands,
               uint32_t rows, uint32_t T, const int64_t* row_ptr, const int32_t* cand,
               int64_t Q, uint16_t* count, uint32_t* bandmask);
int orc_topm_by_count(const int64_t* row_ptr, const int32_t* cand, const uint16_t* count,
                      int64_t Q, int32_t m, int32_t* out_ids, int32_t* out_n);

/* ---- exact Jaccard (Sec. 1) ---- */
double orc_intersection_area(const int32_t* a, int64_t na, const int32_t* b, int64_t nb);
double orc_jaccard(const int32_t* a, int64_t na, const int32_t* b, int64_t nb);

/* ---- reranker MLP reference (fp64, bf16 rounding emulated) ---- */
double orc_bf16_round(double v);
void orc_mlp_forward_backward(const float* x, const float* y, int64_t n_rows,
                              int32_t d_in, int32_t d_h,
                              const double* w1, const double* b1,
                              const double* w2, const double* b2,
                              const double* w3, const double* b3,
                              double* pred, double* loss,
                              double* gw1, double* gb1, double* gw2, double* gb2,
                              double* gw3, double* gb3, int emulate_bf16);

#ifdef __cplusplus
}
#endif
#endif
