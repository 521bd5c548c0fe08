/*
 * oracle.c -- plain CPU oracle for one party's online computation of an
 * actively secure SPDZ2k linear layer with CompactTag (arXiv 2311.04406).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
 * baseline call this file.  It shares no code, header, table or constant with
 * the CUDA library, and the CUDA library never calls it.
 *
 * Every function is the plain definition of the quantity it computes, written
 * as loops over wrapping unsigned __int128 arithmetic reduced mod 2^b, where
 * b = k + s is the share ring width (§2.4: shares and tags live in Z_{2^{k+s}}).
 * Elements are stored row-major as little-endian 64-bit words: one word when
 * b <= 64, two words (lo, hi) when 64 < b <= 128.  Nothing is blocked, fused or
 * reordered: each output element is one sequential sum in index order.  OpenMP
 * only distributes independent output elements over threads.
 *
 * Readings of the paper that this file takes (listed with reasons in the design
 * notes of the repository):
 *   - Eq. (compute-ztag), §2.5: every party adds alpha_i * (E.U) to its tag
 *     share; only party index 0 (the paper's P1) adds E.U to its value share.
 *   - Fig. Pi_OptMAC, §3.2: the tag uses the opened D~ = sum_i [D]_i mod
 *     2^{k+s} (not D mod 2^k).
 *   - Eq. (compute-zcomptag), §3.3: the last term of the compact tag is
 *     alpha_i * E . U^c for every party (the untruncated layer).
 *   - Fig. Pi_CompactMatMul verification: the canonical check share is reduced
 *     mod 2^{k+s}; a separate function keeps the literal mod 2^{k+2s} form.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;
typedef uint64_t u64;
typedef int64_t i64;

static int words_of(int b) { return b <= 64 ? 1 : 2; }

static u128 mask_of(int b) {
    return b >= 128 ? ~(u128)0 : (((u128)1 << b) - 1);
}

static u128 ld(const u64 *p, i64 i, int w) {
    if (w == 1) return (u128)p[i];
    return (u128)p[2 * i] | ((u128)p[2 * i + 1] << 64);
}

static void st(u64 *p, i64 i, int w, u128 v) {
    if (w == 1) { p[i] = (u64)v; return; }
    p[2 * i] = (u64)v;
    p[2 * i + 1] = (u64)(v >> 64);
}

int orc_words(int b) { return words_of(b); }

/* ------------------------------------------------------------------------- */
/* Elementwise ring operations on n elements (§2.4 linearity of shares).     */

void orc_add(int b, i64 n, const u64 *x, const u64 *y, u64 *out) {
    int w = words_of(b); u128 m = mask_of(b);
    for (i64 i = 0; i < n; ++i) st(out, i, w, (ld(x, i, w) + ld(y, i, w)) & m);
}

void orc_sub(int b, i64 n, const u64 *x, const u64 *y, u64 *out) {
    int w = words_of(b); u128 m = mask_of(b);
    for (i64 i = 0; i < n; ++i) st(out, i, w, (ld(x, i, w) - ld(y, i, w)) & m);
}

/* out = c * x, c one ring element */
void orc_smul(int b, i64 n, const u64 *c, const u64 *x, u64 *out) {
    int w = words_of(b); u128 m = mask_of(b); u128 cv = ld(c, 0, w) & m;
    for (i64 i = 0; i < n; ++i) st(out, i, w, (cv * ld(x, i, w)) & m);
}

/* out = x mod 2^b (clears bits above the ring width) */
void orc_reduce(int b, i64 n, const u64 *x, u64 *out) {
    int w = words_of(b); u128 m = mask_of(b);
    for (i64 i = 0; i < n; ++i) st(out, i, w, ld(x, i, w) & m);
}

/* ------------------------------------------------------------------------- */
/* Textbook ring matrix product, §2.2 notation: Out (M x N) = X (M x K) . Y  */
/* (K x N) mod 2^b.  Naive i, j, k loop.                                     */

static u128 dot_col(int w, i64 K, i64 N, const u64 *xrow, const u64 *Y, i64 c) {
    u128 acc = 0;
    for (i64 k = 0; k < K; ++k) acc += ld(xrow, k, w) * ld(Y, k * N + c, w);
    return acc;
}

void orc_ring_gemm(int b, i64 M, i64 K, i64 N, const u64 *X, const u64 *Y, u64 *Out) {
    int w = words_of(b); u128 m = mask_of(b);
    #pragma omp parallel for schedule(static)
    for (i64 r = 0; r < M; ++r)
        for (i64 c = 0; c < N; ++c)
            st(Out, r * N + c, w, dot_col(w, K, N, X + r * K * w, Y, c) & m);
}

/* ------------------------------------------------------------------------- */
/* a1. Share of Z = X.Y from a Beaver matrix triple, Eq. (compute-z) and     */
/* Fig. Pi_MatMul steps 2-3 (§2.5):                                          */
/*   [Z]_i = [C]_i + E.[B]_i + [A]_i.U  (+ E.U for party 0)                  */
/* E = X - A (M x K) and U = Y - B (K x N) are the opened public matrices;   */
/* the paper's U is called F here.                                           */

static u128 share_at(int w, i64 K, i64 N, int party, const u64 *E, const u64 *F,
                     const u64 *A, const u64 *B, const u64 *C, i64 r, i64 c) {
    u128 z = ld(C, r * N + c, w);
    z += dot_col(w, K, N, E + r * K * w, B, c);
    z += dot_col(w, K, N, A + r * K * w, F, c);
    if (party == 0) z += dot_col(w, K, N, E + r * K * w, F, c);
    return z;
}

void orc_linear_share(int b, i64 M, i64 K, i64 N, int party,
                      const u64 *E, const u64 *F, const u64 *A, const u64 *B,
                      const u64 *C, u64 *Z) {
    int w = words_of(b); u128 m = mask_of(b);
    #pragma omp parallel for schedule(static)
    for (i64 r = 0; r < M; ++r)
        for (i64 c = 0; c < N; ++c)
            st(Z, r * N + c, w, share_at(w, K, N, party, E, F, A, B, C, r, c) & m);
}

/* The same share at `cnt` sampled positions (rows[j], cols[j]) -> out[j]. */
void orc_linear_share_at(int b, i64 M, i64 K, i64 N, int party,
                         const u64 *E, const u64 *F, const u64 *A, const u64 *B,
                         const u64 *C, i64 cnt, const i64 *rows, const i64 *cols,
                         u64 *out) {
    int w = words_of(b); u128 m = mask_of(b); (void)M;
    #pragma omp parallel for schedule(static)
    for (i64 j = 0; j < cnt; ++j)
        st(out, j, w, share_at(w, K, N, party, E, F, A, B, C, rows[j], cols[j]) & m);
}

/* ------------------------------------------------------------------------- */
/* a2. Full SPDZ2k tag share, Eq. (compute-ztag), §2.5:                      */
/*   [m(Z)]_i = [m(C)]_i + E.[m(B)]_i + [m(A)]_i.U + [alpha]_i (E.U)         */
/* added by every party.                                                     */

static u128 tag_full_at(int w, i64 K, i64 N, u128 alpha, const u64 *E, const u64 *F,
                        const u64 *mA, const u64 *mB, const u64 *mC, i64 r, i64 c) {
    u128 t = ld(mC, r * N + c, w);
    t += dot_col(w, K, N, E + r * K * w, mB, c);
    t += dot_col(w, K, N, mA + r * K * w, F, c);
    t += alpha * dot_col(w, K, N, E + r * K * w, F, c);
    return t;
}

void orc_linear_tag_full(int b, i64 M, i64 K, i64 N, const u64 *alpha,
                         const u64 *E, const u64 *F, const u64 *mA, const u64 *mB,
                         const u64 *mC, u64 *mZ) {
    int w = words_of(b); u128 m = mask_of(b); u128 a = ld(alpha, 0, w) & m;
    #pragma omp parallel for schedule(static)
    for (i64 r = 0; r < M; ++r)
        for (i64 c = 0; c < N; ++c)
            st(mZ, r * N + c, w, tag_full_at(w, K, N, a, E, F, mA, mB, mC, r, c) & m);
}

void orc_linear_tag_full_at(int b, i64 M, i64 K, i64 N, const u64 *alpha,
                            const u64 *E, const u64 *F, const u64 *mA,
                            const u64 *mB, const u64 *mC, i64 cnt,
                            const i64 *rows, const i64 *cols, u64 *out) {
    int w = words_of(b); u128 m = mask_of(b); u128 a = ld(alpha, 0, w) & m; (void)M;
    #pragma omp parallel for schedule(static)
    for (i64 j = 0; j < cnt; ++j)
        st(out, j, w, tag_full_at(w, K, N, a, E, F, mA, mB, mC, rows[j], cols[j]) & m);
}

/* ------------------------------------------------------------------------- */
/* a3. Optimistic per-element tag, Fig. Pi_OptMAC step 3 (§3.2):             */
/*   [m(Z)]_i = [m(R)]_i - [alpha]_i * D~                                    */

void orc_optmac(int b, i64 M, i64 N, const u64 *alpha, const u64 *mR,
                const u64 *Dt, u64 *mZ) {
    int w = words_of(b); u128 m = mask_of(b); u128 a = ld(alpha, 0, w) & m;
    #pragma omp parallel for schedule(static)
    for (i64 i = 0; i < M * N; ++i)
        st(mZ, i, w, (ld(mR, i, w) - a * ld(Dt, i, w)) & m);
}

/* ------------------------------------------------------------------------- */
/* a4. Compression, Fig. Pi_Compress (§3.1): out (rows) = Mat (rows x cols)  */
/* . chi (cols), a linear combination of the columns.                        */

void orc_compress(int b, i64 rows, i64 cols, const u64 *Mat, const u64 *chi, u64 *out) {
    int w = words_of(b); u128 m = mask_of(b);
    #pragma omp parallel for schedule(static)
    for (i64 r = 0; r < rows; ++r) {
        u128 acc = 0;
        for (i64 c = 0; c < cols; ++c) acc += ld(Mat, r * cols + c, w) * ld(chi, c, w);
        st(out, r, w, acc & m);
    }
}

/* ------------------------------------------------------------------------- */
/* a4 + a5.  Compact tag of the layer, Eq. (compute-zcomptag) (§3.3) with    */
/* the compressions of Fig. Pi_CompactMatMul step 6:                         */
/*   U^c = U.chi, [m(B)^c]_i = [m(B)]_i.chi, [m(C)^c]_i = [m(C)]_i.chi,      */
/*   [m(R)^c]_i = [m(R)]_i.chi, D^c = D~.chi                                 */
/*   [m(Z)^c]_i = [m(C)^c]_i + E.[m(B)^c]_i + [m(A)]_i.U^c                   */
/*                + [alpha]_i (E.U^c)                                        */
/*   [m(D)^c]_i = [m(R)^c]_i - [m(Z)^c]_i                                    */
/* Outputs: Dc (M), mDc (M); mZc (M) when non-NULL.  Returns -1 when the    */
/* host allocation of the intermediate vectors fails.                        */

static int compact_tag(int b, i64 M, i64 K, i64 N, const u64 *alpha,
                       const u64 *E, const u64 *F, const u64 *mA, const u64 *mB,
                       const u64 *mC, const u64 *mR, const u64 *Dt, const u64 *chi,
                       u64 *mDc, u64 *Dc, u64 *mZc, int with_eu) {
    int w = words_of(b); u128 m = mask_of(b); u128 a = ld(alpha, 0, w) & m;
    u128 *scratch = (u128 *)malloc(sizeof(u128) * (size_t)(4 * M + 2 * K + 1));
    if (!scratch) return -1;
    u128 *mRc = scratch;              /* M */
    u128 *mCc = mRc + M;              /* M */
    u128 *Dcv = mCc + M;              /* M */
    u128 *mZcv = Dcv + M;             /* M */
    u128 *mBc = mZcv + M;             /* K */
    u128 *Uc = mBc + K;               /* K */
    for (i64 r = 0; r < M; ++r) {
        u128 s1 = 0, s2 = 0, s3 = 0;
        for (i64 c = 0; c < N; ++c) {
            u128 x = ld(chi, c, w);
            s1 += ld(mR, r * N + c, w) * x;
            s2 += ld(mC, r * N + c, w) * x;
            s3 += ld(Dt, r * N + c, w) * x;
        }
        mRc[r] = s1 & m; mCc[r] = s2 & m; Dcv[r] = s3 & m;
    }
    for (i64 k = 0; k < K; ++k) {
        u128 s1 = 0, s2 = 0;
        for (i64 c = 0; c < N; ++c) {
            u128 x = ld(chi, c, w);
            s1 += ld(mB, k * N + c, w) * x;
            s2 += ld(F, k * N + c, w) * x;
        }
        mBc[k] = s1 & m; Uc[k] = s2 & m;
    }
    for (i64 r = 0; r < M; ++r) {
        u128 e_mb = 0, ma_u = 0, e_u = 0;
        for (i64 k = 0; k < K; ++k) {
            u128 e = ld(E, r * K + k, w);
            e_mb += e * mBc[k];
            ma_u += ld(mA, r * K + k, w) * Uc[k];
            e_u += e * Uc[k];
        }
        mZcv[r] = (mCc[r] + e_mb + ma_u + (with_eu ? a * e_u : 0)) & m;
    }
    for (i64 r = 0; r < M; ++r) {
        st(Dc, r, w, Dcv[r]);
        st(mDc, r, w, (mRc[r] - mZcv[r]) & m);
        if (mZc) st(mZc, r, w, mZcv[r]);
    }
    free(scratch);
    return 0;
}

int orc_compact_tag(int b, i64 M, i64 K, i64 N, const u64 *alpha,
                    const u64 *E, const u64 *F, const u64 *mA, const u64 *mB,
                    const u64 *mC, const u64 *mR, const u64 *Dt, const u64 *chi,
                    u64 *mDc, u64 *Dc, u64 *mZc) {
    return compact_tag(b, M, K, N, alpha, E, F, mA, mB, mC, mR, Dt, chi, mDc, Dc, mZc, 1);
}

/* ------------------------------------------------------------------------- */
/* Truncated layer, Fig. Pi_CompactMatMul with Fig. Pi_OptMAC&Trunc (§3.4).  */
/*                                                                           */
/* Step 2: [Z]_i = [C]_i + E.[B]_i + [A]_i.U for every party (the public     */
/* E.U enters after truncation, step 4).                                     */

void orc_linear_share_trunc(int b, i64 M, i64 K, i64 N, const u64 *E, const u64 *F,
                            const u64 *A, const u64 *B, const u64 *C, u64 *Z) {
    orc_linear_share(b, M, K, N, 1, E, F, A, B, C, Z);   /* a party index > 0 adds no E.U */
}

/* Steps 3-4 (Pi_OptMAC&Trunc steps 3-4, then P1's public term):            */
/*   delta = D / 2^f with D = D~ mod 2^k, rho = (E.U mod 2^k) / 2^f          */
/*   (both floor divisions of the k-bit value), tau = rho - delta;           */
/*   [Z^f]_i = [R^f]_i + tau (party 0 only; a public constant is added once)  */
/*   [m(Z^f)]_i = [m(R^f)]_i + [alpha]_i * tau (every party).                */
/* P is the public product E.U (M x N, mod 2^{k+s}).                         */
void orc_optmac_trunc(int k, int s, i64 M, i64 N, int f, int party, const u64 *alpha,
                      const u64 *Rf, const u64 *mRf, const u64 *Dt, const u64 *P,
                      u64 *Zf, u64 *mZf) {
    int b = k + s;
    int w = words_of(b); u128 m = mask_of(b); u128 mk = mask_of(k);
    u128 a = ld(alpha, 0, w) & m;
    #pragma omp parallel for schedule(static)
    for (i64 i = 0; i < M * N; ++i) {
        u128 delta = (ld(Dt, i, w) & mk) >> f;
        u128 rho = (ld(P, i, w) & mk) >> f;
        u128 tau = (rho - delta) & m;
        st(Zf, i, w, (ld(Rf, i, w) + (party == 0 ? tau : 0)) & m);
        st(mZf, i, w, (ld(mRf, i, w) + a * tau) & m);
    }
}

/* Steps 6-7: the compact tag without an E.U^c term,                         */
/*   [m(Z)^c]_i = [m(C)^c]_i + E.[m(B)^c]_i + [m(A)]_i.U^c,                  */
/*   [m(D)^c]_i = [m(R)^c]_i - [m(Z)^c]_i, D^c = D~.chi.                     */
int orc_compact_tag_trunc(int b, i64 M, i64 K, i64 N, const u64 *alpha,
                          const u64 *E, const u64 *F, const u64 *mA, const u64 *mB,
                          const u64 *mC, const u64 *mR, const u64 *Dt, const u64 *chi,
                          u64 *mDc, u64 *Dc, u64 *mZc) {
    return compact_tag(b, M, K, N, alpha, E, F, mA, mB, mC, mR, Dt, chi, mDc, Dc, mZc, 0);
}

/* ------------------------------------------------------------------------- */
/* a6. Check share of the compact verification, Fig. Pi_CompactMatMul        */
/* verification steps 3-5, reduced mod 2^{k+s} (canonical reading):          */
/*   cs_i = sum_r chi^_r * ([alpha]_i * D^c_r - [m(D)^c]_{i,r})              */

void orc_check_compact(int b, i64 M, const u64 *alpha, const u64 *chi_hat,
                       const u64 *Dc, const u64 *mDc, u64 *cs) {
    int w = words_of(b); u128 m = mask_of(b); u128 a = ld(alpha, 0, w) & m;
    u128 acc = 0;
    for (i64 r = 0; r < M; ++r)
        acc += ld(chi_hat, r, w) * (a * ld(Dc, r, w) - ld(mDc, r, w));
    st(cs, 0, w, acc & m);
}

/* The same check in the printed modulus 2^{k+2s}: step 3 reduces
 * [alpha]_i * D^c mod 2^{k+s}; steps 4-5 multiply by chi^ and sum mod
 * 2^{k+2s}.  Only defined for k + 2s <= 128; the result is two words. */
int orc_check_compact_literal(int k, int s, i64 M, const u64 *alpha, const u64 *chi_hat,
                              const u64 *Dc, const u64 *mDc, u64 *cs2) {
    int b = k + s;
    if (k + 2 * s > 128) return -1;
    int w = words_of(b); u128 m = mask_of(b); u128 m2 = mask_of(k + 2 * s);
    u128 a = ld(alpha, 0, w) & m;
    u128 acc = 0;
    for (i64 r = 0; r < M; ++r) {
        u128 CS = (a * ld(Dc, r, w)) & m;
        u128 x = ld(chi_hat, r, w);
        acc += CS * x - ld(mDc, r, w) * x;
    }
    acc &= m2;
    cs2[0] = (u64)acc; cs2[1] = (u64)(acc >> 64);
    return 0;
}

/* Tag-check share of Fig. Pi_BatchRec (§2.5), tag check steps 2-3:
 *   cs_i = sum_{p,q} ( [m(W)]_{i,pq} chi_pq - [alpha]_i (W_pq chi_pq) )      */
void orc_check_batchrec(int b, i64 M, i64 N, const u64 *alpha, const u64 *chi,
                        const u64 *W, const u64 *mW, u64 *cs) {
    int w = words_of(b); u128 m = mask_of(b); u128 a = ld(alpha, 0, w) & m;
    u128 acc = 0;
    for (i64 i = 0; i < M * N; ++i) {
        u128 x = ld(chi, i, w);
        acc += ld(mW, i, w) * x - a * (ld(W, i, w) * x);
    }
    st(cs, 0, w, acc & m);
}

/* ------------------------------------------------------------------------- */
/* Pi_BatchRec (§2.5), open phase step 1 for an opened difference V = X - A:   */
/*   [W]_i = [X]_i - [A]_i + [R]_i,  [m(W)]_i = [m(X)]_i - [m(A)]_i + [m(R)]_i  */
/* where R is a sharing of a matrix that is 0 mod 2^k.  A and mA may be NULL  */
/* (then V = X).                                                             */
void orc_batchrec_mask(int b, i64 n, const u64 *X, const u64 *A, const u64 *R,
                       const u64 *mX, const u64 *mA, const u64 *mR, u64 *W, u64 *mW) {
    int w = words_of(b); u128 m = mask_of(b);
    for (i64 i = 0; i < n; ++i) {
        u128 v = ld(X, i, w) - (A ? ld(A, i, w) : 0) + ld(R, i, w);
        u128 t = ld(mX, i, w) - (mA ? ld(mA, i, w) : 0) + ld(mR, i, w);
        st(W, i, w, v & m);
        st(mW, i, w, t & m);
    }
}

/* Public combiners from a coin-tossed seed (F_Rand, App. A.1, expanded by a */
/* PRG): the SplitMix64 sequence (Steele, Lea & Flood 2014) whose state starts */
/* at `seed`: chi_i = mix(seed + (i + 1) GAMMA) mod 2^s, s <= 64, with        */
/* mix(z): z = (z ^ (z >> 30)) C1; z = (z ^ (z >> 27)) C2; z ^ (z >> 31).     */
static u64 splitmix_mix(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void orc_chi_seeded(int b, int s, u64 seed, i64 n, u64 *out) {
    int w = words_of(b);
    const u64 g = 0x9E3779B97F4A7C15ULL;
    u128 ms = mask_of(s);
    for (i64 i = 0; i < n; ++i)
        st(out, i, w, (u128)splitmix_mix(seed + (u64)(i + 1) * g) & ms);
}


/* Threads of the OpenMP loops (for timing the oracle on one core or on all of
 * them); n <= 0 leaves the setting alone.  Returns the previous maximum. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    const int old = omp_get_max_threads();
    if (n > 0) omp_set_num_threads(n);
    return old;
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* im2col view of a convolution (§2.6): row (b, oy, ox), column (c, ky, kx)  */
/* of the output is in[b][c][oy*stride + ky - pad][ox*stride + kx - pad]    */
/* (NCHW input), or 0 in the zero padding.  Output rows B*Ho*Wo, columns     */
/* C*f*f, with Ho = (H - f + 2 pad) / stride + 1 and Wo likewise.            */
void orc_im2col(int words, int64_t B, int64_t C, int64_t H, int64_t W, int f, int pad, int stride,
                const uint64_t *in, uint64_t *out) {
    const int64_t Ho = (H - f + 2 * pad) / stride + 1, Wo = (W - f + 2 * pad) / stride + 1;
    const int64_t cols = C * f * f;
    for (int64_t b = 0; b < B; ++b)
        for (int64_t oy = 0; oy < Ho; ++oy)
            for (int64_t ox = 0; ox < Wo; ++ox) {
                const int64_t row = (b * Ho + oy) * Wo + ox;
                for (int64_t c = 0; c < C; ++c)
                    for (int ky = 0; ky < f; ++ky)
                        for (int kx = 0; kx < f; ++kx) {
                            const int64_t col = (c * f + ky) * f + kx;
                            const int64_t y = oy * stride + ky - pad, x = ox * stride + kx - pad;
                            for (int h = 0; h < words; ++h) {
                                uint64_t v = 0;
                                if (y >= 0 && y < H && x >= 0 && x < W)
                                    v = in[(((b * C + c) * H + y) * W + x) * words + h];
                                out[(row * cols + col) * words + h] = v;
                            }
                        }
            }
}
