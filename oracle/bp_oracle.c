/*
 * bp_oracle.c -- plain, slow, FP64 CPU oracle for the event-driven spiking
 * network hot path of BrainPy (Wang et al., "A differentiable brain simulator
 * bridging brain simulation and brain-inspired computing", ICLR 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or constant generator with the CUDA library: every
 * formula below is written out again from the paper (and, for the random
 * number generators, from their published definitions).
 *
 * Every routine is a straight loop in the order the paper states the
 * computation; nothing is blocked, fused or reordered.  Floating point is FP64
 * throughout; integer event counts are exact.
 *
 * Readings of the paper that this file fixes (the paper is silent or
 * inconsistent at these points):
 *   R1  Appendix B pseudo-code adds data[j] at outs[indices[i]]; the loop over
 *       j only makes sense as outs[indices[j]].
 *   R2  The stored matrix is presynaptic-row-major: rows are walked by event
 *       index, so the event product is the scatter y = W^T s, and its
 *       "transpose" is the gather y_pre = W x.
 *   R3  Appendix C seeds one sequential stream; here row i draws from its own
 *       counter-based stream so that a row is the same at every call whatever
 *       else spiked (the reproducibility the appendix asks of the seed).
 *       Draw k of row i for stream s is word (k mod 4) of
 *       Philox4x32-10(key = seed, counter = (k div 4, i, s, 0)).
 *   R4  Gap range K = ceil(2/p - 1) (the executable form; the prose writes a
 *       floor; both agree when 2/p is an integer).  K >= 1.
 *   R5  First target is U[1,K] - 1 (zero-based); later targets add U[1,K].
 *   R6  U[1,K] = 1 + floor(x * K / 2^32) for a 32-bit draw x.
 *   R7  Self-connections are allowed (the generator does not exclude them).
 *   R9  Within a step: synaptic decay, then add the events delivered by the
 *       previous step's spikes; the COBA current uses the membrane potential
 *       from before this step's update; spikes of this step are delivered at
 *       the next step.
 *   R10 Exponential Euler holds the input current fixed over the step.
 *   R11 Spike when V > V_th (strict).
 *   R12 tau_ref / dt refractory steps held as an integer counter; V stays at
 *       the reset value, conductances keep decaying and integrating.
 */
#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from Salmon, Moraes, Dror and Shaw, "Parallel random        */
/* numbers: as easy as 1, 2, 3" (SC 2011): ten rounds of two 32x32->64 bit    */
/* multiplies whose high/low halves are permuted and xored with the counter   */
/* words and the round key; the key is bumped by the Weyl constants between  */
/* rounds.                                                                     */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014): the j-th  */
/* output (j = 0, 1, ...) of the generator started at state s.                */
uint64_t orc_splitmix64(uint64_t s, uint64_t j)
{
    uint64_t z = s + (j + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Projection seeds of the E/I network: excitatory rows use output 0 and     */
/* inhibitory rows output 1 of SplitMix64 started at the network seed.       */
uint64_t orc_projection_seed(uint64_t net_seed, int projection)
{
    return orc_splitmix64(net_seed, (uint64_t)projection);
}

/* One 32-bit draw of row `row`, stream `stream`, index k (reading R3). */
uint32_t orc_jit_draw(uint64_t seed, uint32_t row, uint32_t stream, uint64_t k)
{
    uint32_t ctr[4] = {(uint32_t)(k >> 2), row, stream, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[k & 3u];
}

/* Appendix C: gap range K so that E[U[1,K]] = (K+1)/2 = 1/p (reading R4).  */
/* The relative guard absorbs the representation error of p = a/b so that   */
/* 2/p - 1 lands on the integer it denotes.                                  */
int64_t orc_jit_K(double p)
{
    double x = 2.0 / p - 1.0;
    double k = ceil(x - 1e-12 * fabs(x));
    if (k < 1.0) k = 1.0;
    return (int64_t)k;
}

/* Weight kinds shared by the JIT generator's callers. */
enum { ORC_W_HOMO = 0, ORC_W_UNIFORM = 1, ORC_W_NORMAL = 2 };

/* Gap U[1,K] from one draw (reading R6). */
static int64_t orc_gap(uint64_t seed, uint32_t row, uint64_t k, int64_t K)
{
    uint64_t x = orc_jit_draw(seed, row, 0u, k);
    return 1 + (int64_t)((x * (uint64_t)K) >> 32);
}

/* Weight of the k-th synapse of a row.  Uniform: w0 + (w1 - w0) u with       */
/* u = (x >> 8) 2^-24 in [0,1) from stream 1.  Normal: mean w0, std w1, one   */
/* Box-Muller cosine branch per synapse from the two words (2(k mod 2),       */
/* 2(k mod 2)+1) of the stream-2 block k div 2, with u1 in (0,1].            */
double orc_jit_weight(uint64_t seed, uint32_t row, uint64_t k, int wkind, double w0, double w1)
{
    if (wkind == ORC_W_HOMO) return w0;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    if (wkind == ORC_W_UNIFORM) {
        uint32_t ctr[4] = {(uint32_t)(k >> 2), row, 1u, 0u};
        orc_philox4x32_10(ctr, key, out);
        double u = (double)(out[k & 3u] >> 8) * (1.0 / 16777216.0);
        return w0 + (w1 - w0) * u;
    }
    uint32_t ctr[4] = {(uint32_t)(k >> 1), row, 2u, 0u};
    orc_philox4x32_10(ctr, key, out);
    uint32_t a = out[2u * (k & 1u)], b = out[2u * (k & 1u) + 1u];
    double u1 = (double)((a >> 8) + 1u) * (1.0 / 16777216.0);
    double u2 = (double)(b >> 8) * (1.0 / 16777216.0);
    double z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    return w0 + w1 * z;
}

/* Appendix C: postsynaptic targets (and weights) of presynaptic row `row`.  */
/* Writes at most `cap` entries, returns the row length.                     */
int64_t orc_jit_row(uint64_t seed, int64_t K, int wkind, double w0, double w1, uint32_t row,
                    int64_t n_post, int32_t* cols, double* w, int64_t cap)
{
    int64_t n = 0;
    uint64_t k = 0;
    int64_t q = orc_gap(seed, row, 0, K) - 1;       /* reading R5 */
    while (q < n_post) {
        if (n < cap) {
            if (cols) cols[n] = (int32_t)q;
            if (w) w[n] = orc_jit_weight(seed, row, k, wkind, w0, w1);
        }
        ++n;
        ++k;
        q += orc_gap(seed, row, k, K);
    }
    return n;
}

/* Appendix C pseudo-code as an operator: y[target] += weight for every      */
/* target of every row whose event flag is set.                              */
void orc_jitconn_event_mv(uint64_t seed, int64_t K, int wkind, double w0, double w1,
                          int64_t n_pre, int64_t n_post, const uint8_t* events, double* y)
{
    for (int64_t i = 0; i < n_pre; ++i) {
        if (!events[i]) continue;
        uint64_t k = 0;
        int64_t q = orc_gap(seed, (uint32_t)i, 0, K) - 1;
        while (q < n_post) {
            y[q] += orc_jit_weight(seed, (uint32_t)i, k, wkind, w0, w1);
            ++k;
            q += orc_gap(seed, (uint32_t)i, k, K);
        }
    }
}

/* Non-event JIT product with a dense vector: y[target] += w * x[row]. */
void orc_jitconn_mv(uint64_t seed, int64_t K, int wkind, double w0, double w1,
                    int64_t n_pre, int64_t n_post, const double* x, double* y)
{
    for (int64_t i = 0; i < n_pre; ++i) {
        uint64_t k = 0;
        int64_t q = orc_gap(seed, (uint32_t)i, 0, K) - 1;
        while (q < n_post) {
            y[q] += orc_jit_weight(seed, (uint32_t)i, k, wkind, w0, w1) * x[i];
            ++k;
            q += orc_gap(seed, (uint32_t)i, k, K);
        }
    }
}

/* Transposed JIT product: y_pre[row] = sum over the row's targets of w x[target]. */
void orc_jitconn_mv_t(uint64_t seed, int64_t K, int wkind, double w0, double w1,
                      int64_t n_pre, int64_t n_post, const double* x, double* y_pre)
{
    for (int64_t i = 0; i < n_pre; ++i) {
        uint64_t k = 0;
        double acc = 0.0;
        int64_t q = orc_gap(seed, (uint32_t)i, 0, K) - 1;
        while (q < n_post) {
            acc += orc_jit_weight(seed, (uint32_t)i, k, wkind, w0, w1) * x[q];
            ++k;
            q += orc_gap(seed, (uint32_t)i, k, K);
        }
        y_pre[i] += acc;
    }
}

/* Row lengths of the JIT matrix (first pass of materialising it as CSR). */
void orc_jit_row_lengths(uint64_t seed, int64_t K, int64_t n_pre, int64_t n_post, int64_t* len)
{
    for (int64_t i = 0; i < n_pre; ++i)
        len[i] = orc_jit_row(seed, K, ORC_W_HOMO, 0.0, 0.0, (uint32_t)i, n_post, NULL, NULL, 0);
}

/* ------------------------------------------------------------------------ */
/* Appendix B: event-driven CSR product (reading R1, R2).  data == NULL      */
/* means every stored entry has the homogeneous value w_homo.                */
/* ------------------------------------------------------------------------ */
void orc_event_csrmv(int64_t n_pre, const int64_t* indptr, const int32_t* indices, const double* data,
                     double w_homo, const uint8_t* events, double* y)
{
    for (int64_t i = 0; i < n_pre; ++i) {
        if (!events[i]) continue;
        for (int64_t j = indptr[i]; j < indptr[i + 1]; ++j)
            y[indices[j]] += data ? data[j] : w_homo;
    }
}

/* Integer event counts: the homogeneous-weight product before the weight   */
/* is applied, c[post] += 1 per delivered event.                            */
void orc_event_csr_count(int64_t n_pre, const int64_t* indptr, const int32_t* indices,
                         const uint8_t* events, int64_t* c)
{
    for (int64_t i = 0; i < n_pre; ++i) {
        if (!events[i]) continue;
        for (int64_t j = indptr[i]; j < indptr[i + 1]; ++j) c[indices[j]] += 1;
    }
}

/* Gather form over the same rows: y_pre[i] += sum_j W[i, j] x[j]. */
void orc_csrmv_t(int64_t n_pre, const int64_t* indptr, const int32_t* indices, const double* data,
                 double w_homo, const double* x, double* y_pre)
{
    for (int64_t i = 0; i < n_pre; ++i) {
        double acc = 0.0;
        for (int64_t j = indptr[i]; j < indptr[i + 1]; ++j)
            acc += (data ? data[j] : w_homo) * x[indices[j]];
        y_pre[i] += acc;
    }
}

/* Reverse mode of the event product with respect to the stored weights:   */
/* dW[j] += s[i] * delta[indices[j]] for every entry j of row i.             */
void orc_event_csrmv_dw(int64_t n_pre, const int64_t* indptr, const int32_t* indices,
                        const uint8_t* events, const double* delta, double* dw)
{
    for (int64_t i = 0; i < n_pre; ++i) {
        if (!events[i]) continue;
        for (int64_t j = indptr[i]; j < indptr[i + 1]; ++j) dw[j] += delta[indices[j]];
    }
}

/* ------------------------------------------------------------------------ */
/* COBA E/I network of LIF neurons with exponential conductance synapses.   */
/*   Appendix E: g <- exp(-dt/tau) g, then g <- g + w per delivered spike.  */
/*   Appendix F: tau dV/dt = -(V - V_rest) + R G,  G = -sum g (V - E),       */
/*               spike when V > V_th, then V <- V_reset.                     */
/*   Appendix N, Listing S6: E rows project with weight w_e (E = 0 mV,       */
/*               tau = 5 ms), I rows with w_i (E = -80 mV, tau = 10 ms), one  */
/*               merged conductance per postsynaptic neuron and type, the   */
/*               previous step's spikes are delivered, input 20 each step.  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n, n_e;
    double dt, tau_m, tau_e, tau_i;
    double V_rest, V_th, V_reset, E_e, E_i, R, I_ext;
    double w_e, w_i;
    int32_t ref_steps;
} orc_coba;

/* Connectivity of the network.  kind 0: one CSR over all n presynaptic rows */
/* (data NULL = homogeneous w_e / w_i, delivered as integer counts).         */
/* kind 1: JIT rows, E rows 0..n_e-1 with seed_e, I rows 0..n-n_e-1 with     */
/* seed_i, homogeneous weights.                                              */
typedef struct {
    int32_t kind;
    const int64_t* indptr;
    const int32_t* indices;
    const double* data;
    uint64_t seed_e, seed_i;
    int64_t K;
} orc_conn;

/* One time step.  ye / yi hold what the previous step delivered (counts in */
/* the homogeneous case, weighted sums otherwise) and receive this step's    */
/* deliveries.  Returns the number of spikes; spk[i] is set to 0/1.  vdec    */
/* (nullable) receives the potential the threshold test saw (NAN while      */
/* refractory), so callers can tell how close each decision was.            */
int64_t orc_coba_step(const orc_coba* P, const orc_conn* C, double* V, double* ge, double* gi,
                      int32_t* ref, double* ye, double* yi, uint8_t* spk, double* vdec)
{
    const double a_m = exp(-P->dt / P->tau_m);
    const double a_e = exp(-P->dt / P->tau_e);
    const double a_i = exp(-P->dt / P->tau_i);
    const int homo = (C->kind == 1) || (C->data == NULL);
    int64_t n_spk = 0;
    for (int64_t i = 0; i < P->n; ++i) {
        /* synapses: decay, then the delivered events (R9) */
        double add_e = homo ? P->w_e * ye[i] : ye[i];
        double add_i = homo ? P->w_i * yi[i] : yi[i];
        ge[i] = ge[i] * a_e + add_e;
        gi[i] = gi[i] * a_i + add_i;
        ye[i] = 0.0;
        yi[i] = 0.0;
        /* COBA current with the pre-update potential */
        double I = ge[i] * (P->E_e - V[i]) + gi[i] * (P->E_i - V[i]) + P->I_ext;
        spk[i] = 0;
        if (vdec) vdec[i] = NAN;
        if (ref[i] > 0) {
            ref[i] -= 1; /* R12: clamped, V unchanged */
            continue;
        }
        /* R10: exact solution of the linear ODE with I held over the step */
        double V_inf = P->V_rest + P->R * I;
        V[i] = V_inf + (V[i] - V_inf) * a_m;
        if (vdec) vdec[i] = V[i];
        if (V[i] > P->V_th) { /* R11 */
            spk[i] = 1;
            V[i] = P->V_reset;
            ref[i] = P->ref_steps;
            ++n_spk;
        }
    }
    /* deliver this step's spikes (Appendix B / C), E rows into ye, I rows into yi */
    for (int64_t i = 0; i < P->n; ++i) {
        if (!spk[i]) continue;
        const int is_e = i < P->n_e;
        double* y = is_e ? ye : yi;
        if (C->kind == 0) {
            for (int64_t j = C->indptr[i]; j < C->indptr[i + 1]; ++j)
                y[C->indices[j]] += C->data ? C->data[j] : 1.0;
        } else {
            uint64_t seed = is_e ? C->seed_e : C->seed_i;
            uint32_t row = (uint32_t)(is_e ? i : i - P->n_e);
            int64_t q = orc_gap(seed, row, 0, C->K) - 1;
            uint64_t k = 0;
            while (q < P->n) {
                y[q] += 1.0;
                ++k;
                q += orc_gap(seed, row, k, C->K);
            }
        }
    }
    return n_spk;
}

/* T steps.  Per-step spike counts of the E and I populations go to         */
/* spikes_e / spikes_i (length T, nullable); raster (T x n, nullable) gets   */
/* the spike flags; events (length T, nullable) the number of synaptic       */
/* events each step delivered.                                               */
void orc_coba_run(const orc_coba* P, const orc_conn* C, int64_t T, double* V, double* ge, double* gi,
                  int32_t* ref, double* ye, double* yi, int64_t* spikes_e, int64_t* spikes_i,
                  int64_t* events, uint8_t* raster)
{
    uint8_t* spk = (uint8_t*)malloc((size_t)P->n);
    for (int64_t t = 0; t < T; ++t) {
        orc_coba_step(P, C, V, ge, gi, ref, ye, yi, spk, NULL);
        int64_t ne = 0, ni = 0, ev = 0;
        for (int64_t i = 0; i < P->n; ++i) {
            if (!spk[i]) continue;
            if (i < P->n_e) ++ne; else ++ni;
            if (events) {
                if (C->kind == 0) {
                    ev += C->indptr[i + 1] - C->indptr[i];
                } else {
                    int is_e = i < P->n_e;
                    ev += orc_jit_row(is_e ? C->seed_e : C->seed_i, C->K, ORC_W_HOMO, 0, 0,
                                      (uint32_t)(is_e ? i : i - P->n_e), P->n, NULL, NULL, 0);
                }
            }
        }
        if (spikes_e) spikes_e[t] = ne;
        if (spikes_i) spikes_i[t] = ni;
        if (events) events[t] = ev;
        if (raster) memcpy(raster + t * P->n, spk, (size_t)P->n);
    }
    free(spk);
}

/* Population rate in Hz from a spike total over n neurons and T steps of   */
/* dt milliseconds.                                                          */
double orc_rate_hz(int64_t total_spikes, int64_t n, int64_t T, double dt_ms)
{
    return (double)total_spikes / ((double)n * (double)T * dt_ms * 1e-3);
}
