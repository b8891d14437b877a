/*
 * oracle.c -- plain, slow, FP64 CPU oracle of SimNet's sub-trace simulation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file:
 * only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg load it.  It shares no code, header, table or constant with the CUDA
 * library; both sides only read the same packed instruction records.
 *
 * What it computes (SimNet, arXiv 2105.05821):
 *   - the 50-feature rows of the current instruction and its context
 *     instructions (Sec. 2.2, Table 1, in the synthetic encoding below);
 *   - the CNN latency predictor: k=2 / stride-2 convolutions with ReLU, or
 *     residual blocks (the RB models), flatten, FC + ReLU, FC to the
 *     latencies (Sec. 2.3, Fig. 2);
 *   - latency = softplus(output), clamped to [0, 255] and rounded half-to-even;
 *     or, with the hybrid head (Sec. 2.3), per latency the class with the
 *     largest of 10 logits (0..8 cycles, or "more than 8", which takes the
 *     regression output as above);
 *   - the processor queue and curTick clock: fetch latency advances curTick,
 *     in-order retire when residence reaches the execution latency, retire
 *     bandwidth, eviction at capacity, append with residence 0, and the drain
 *     after the last instruction (Sec. 3.2), so that the final curTick equals
 *     the sum of fetch latencies plus Delta (Sec. 3.1, Eq. 1);
 *   - optionally a third latency, the store latency, and the memory write
 *     queue: a store that retires from the processor queue enters it and
 *     leaves, in order and with no bandwidth limit, once its residence reaches
 *     the store latency (Sec. 3.2);
 *   - sub-traces simulated independently, each from an empty queue and
 *     curTick = 0 (Sec. 3.3);
 *   - the MSE training loss (hybrid head: cross-entropy of the class logits
 *     plus the squared error of the regression output), its analytic FP64
 *     gradient and an Adam step (Sec. 2.4).
 *
 * Readings taken where the paper is silent (each also listed in the design
 * notes): L = W rows (current + W-1 context) and queue capacity W-1; an
 * entry is ready when residence >= E (strict '>' selectable); the retire
 * budget over a jump of F cycles is retire_width * F and none when F = 0, the
 * drain advances one cycle at a time with budget retire_width; a full queue
 * evicts its oldest entry; NaN latencies become 255.
 *
 * Feature encoding of one row (channel: meaning):
 *   0-31 opcode one-hot | 32,33,34 src0/32, src1/32, dst/32 |
 *   35,36,37 is_load, is_store, is_branch | 38-40 cache level one-hot |
 *   41 mispredict | 42 min(residence, 4095)/64 | 43 E/64 |
 *   44 S/64 for a store when the memory write queue is modelled, else 0 |
 *   45,46,47 ctx.dst == cur.src0 / cur.src1 / cur.dst |
 *   48 both are memory ops at the same cache level | 49 zero.
 * The current instruction's row keeps channels 42-49 at zero (the paper pads
 * its 47 current-instruction features with three zeros, Sec. 2.2).
 *
 * parity pins: see tests/test_oracle_*.py (hand-stepped traces, closed forms,
 * invariants, torch float64 conv1d/linear, finite differences).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NF 50            /* features per row (Sec. 2.2) */
#define MAXCONV 8

typedef struct {
    int32_t window;        /* W: rows given to the CNN */
    int32_t n_conv;        /* k=2, s=2 conv layers */
    int32_t channels;      /* conv output channels */
    int32_t hidden;        /* FC1 width */
    int32_t retire_width;  /* processor-queue retire bandwidth per cycle */
    int32_t retire_strict; /* 0: ready at residence >= E; 1: residence > E */
    int32_t hybrid;        /* 0: regression head; 1: hybrid head (11 outputs per latency) */
    int32_t store_queue;   /* 1: a third latency (store) and the memory write queue (Sec. 3.2) */
    int32_t residual;      /* 1: the n_conv layers are residual blocks (RB models, Sec. 2.3) */
} oracle_cfg;

/* Latencies predicted per instruction: fetch, execution (and store). */
static int n_lat(const oracle_cfg *c) { return c->store_queue ? 3 : 2; }
/* FC2 outputs: regression, one per latency [fetch, execution(, store)]; hybrid,
 * per latency t: 10 class logits (0..8 cycles, "more than 8") then one value. */
static int n_out(const oracle_cfg *c) { return (c->hybrid ? 11 : 1) * n_lat(c); }
#define MAXOUT 33

/* ------------------------------------------------------------------ records */
typedef struct { int op, s0, s1, dst, ld, st, br, lvl, mp; } inst_t;

static inst_t decode(uint32_t r)
{
    inst_t a;
    a.op = (int)(r & 31u);
    a.s0 = (int)((r >> 5) & 31u);
    a.s1 = (int)((r >> 10) & 31u);
    a.dst = (int)((r >> 15) & 31u);
    a.ld = (int)((r >> 20) & 1u);
    a.st = (int)((r >> 21) & 1u);
    a.br = (int)((r >> 22) & 1u);
    a.lvl = (int)((r >> 23) & 3u);
    a.mp = (int)((r >> 25) & 1u);
    return a;
}

/* ------------------------------------------------------------------ features (Sec. 2.2) */
static void encode_static(const inst_t *a, double *row)
{
    row[a->op] = 1.0;
    row[32] = a->s0 / 32.0;
    row[33] = a->s1 / 32.0;
    row[34] = a->dst / 32.0;
    row[35] = a->ld;
    row[36] = a->st;
    row[37] = a->br;
    row[38 + a->lvl] = 1.0;
    row[41] = a->mp;
}

/* One context row: static features, residence, execution latency and (for a
 * store, with the memory write queue modelled) store latency, and the
 * dependency flags against the current instruction. */
static void encode_context(const inst_t *cur, uint32_t ctx_rec, int64_t residence, int e, int s,
                           double *row)
{
    inst_t c = decode(ctx_rec);
    encode_static(&c, row);
    if (residence > 4095) residence = 4095;
    row[42] = (double)residence / 64.0;
    row[43] = e / 64.0;
    row[44] = c.st ? s / 64.0 : 0.0;
    row[45] = (c.dst == cur->s0);
    row[46] = (c.dst == cur->s1);
    row[47] = (c.dst == cur->dst);
    row[48] = ((c.ld || c.st) && (cur->ld || cur->st) && c.lvl == cur->lvl);
    row[49] = 0.0;
}

/* ------------------------------------------------------------------ CNN (Sec. 2.3) */
/* Layer k of a residual network is a residual block (the paper draws it only
 * in a figure; this build's reading, in the spirit of the EfficientNet-style
 * blocks it cites, with the kernel-2 / stride-2 rule kept):
 *   a = ReLU(conv_k(x)), k = 2, stride 2, with bias (cw, cb);
 *   y = ReLU(pw_k(a) + proj_k(x)), pw a pointwise (k = 1) conv with bias (pw,
 *   pwb) and proj a k = 2 / stride-2 conv without bias (pj), the shortcut that
 *   matches the halved length and the channel count.
 * Blob order per block: conv.weight [C][Cin][2], conv.bias [C], pw.weight
 * [C][C][1], pw.bias [C], proj.weight [C][Cin][2]. */
typedef struct {
    const double *cw[MAXCONV], *cb[MAXCONV];
    const double *pw[MAXCONV], *pwb[MAXCONV], *pj[MAXCONV];   /* residual blocks only */
    const double *w1, *b1, *w2, *b2;
} net_t;

static int64_t blob_size(const oracle_cfg *c)
{
    int64_t n = 0, cin = NF;
    for (int k = 0; k < c->n_conv; k++) {
        n += (int64_t)c->channels * cin * 2 + c->channels;
        if (c->residual) n += (int64_t)c->channels * c->channels + c->channels + (int64_t)c->channels * cin * 2;
        cin = c->channels;
    }
    int64_t fin = (int64_t)c->channels * (c->window >> c->n_conv);
    n += fin * c->hidden + c->hidden + (int64_t)n_out(c) * c->hidden + n_out(c);
    return n;
}

static net_t net_view(const oracle_cfg *c, const double *blob)
{
    net_t n;
    const double *p = blob;
    int cin = NF;
    for (int k = 0; k < c->n_conv; k++) {
        n.cw[k] = p; p += (int64_t)c->channels * cin * 2;
        n.cb[k] = p; p += c->channels;
        if (c->residual) {
            n.pw[k] = p; p += (int64_t)c->channels * c->channels;
            n.pwb[k] = p; p += c->channels;
            n.pj[k] = p; p += (int64_t)c->channels * cin * 2;
        }
        cin = c->channels;
    }
    int64_t fin = (int64_t)c->channels * (c->window >> c->n_conv);
    n.w1 = p; p += fin * c->hidden;
    n.b1 = p; p += c->hidden;
    n.w2 = p; p += (int64_t)n_out(c) * c->hidden;
    n.b2 = p;
    return n;
}

/* Work area holding every layer's output, kept for the backward pass. */
typedef struct {
    double *act[MAXCONV + 1];  /* act[0] = input [W][NF]; act[k+1] = conv k out [W>>(k+1)][C] */
    double *ra, *rs;           /* residual blocks: branch and shortcut [W/2][C] (reused per block) */
    double *hid;               /* FC1 output after ReLU [H] */
    double z[MAXOUT];          /* FC2 outputs (before softplus / class decision) */
} fwd_t;

static size_t fwd_doubles(const oracle_cfg *c)
{
    size_t n = (size_t)c->window * NF;
    for (int k = 0; k < c->n_conv; k++) n += (size_t)(c->window >> (k + 1)) * c->channels;
    if (c->residual) n += 2 * (size_t)(c->window >> 1) * c->channels;
    return n + c->hidden;
}

static void fwd_bind(const oracle_cfg *c, double *mem, const double *x, fwd_t *f)
{
    f->act[0] = (double *)x;
    double *p = mem;
    for (int k = 0; k < c->n_conv; k++) {
        f->act[k + 1] = p;
        p += (size_t)(c->window >> (k + 1)) * c->channels;
    }
    f->ra = f->rs = NULL;
    if (c->residual) {
        f->ra = p;
        p += (size_t)(c->window >> 1) * c->channels;
        f->rs = p;
        p += (size_t)(c->window >> 1) * c->channels;
    }
    f->hid = p;
}

/* y[l][co] = ReLU(b[co] + sum_{ci, t in {0,1}} W[co][ci][t] * x[2l+t][ci])  (k = 2, stride 2) */
static void conv_forward(const double *w, const double *b, const double *x, int rows_in, int cin,
                         int cout, double *y)
{
    for (int l = 0; l < rows_in / 2; l++)
        for (int co = 0; co < cout; co++) {
            double s = b[co];
            for (int ci = 0; ci < cin; ci++)
                for (int t = 0; t < 2; t++)
                    s += w[((int64_t)co * cin + ci) * 2 + t] * x[(int64_t)(2 * l + t) * cin + ci];
            y[(int64_t)l * cout + co] = s > 0.0 ? s : 0.0;
        }
}

/* Residual block k: a = ReLU(conv(x)); s = proj(x); y = ReLU(pw(a) + pw bias + s). */
static void residual_forward(const net_t *n, int k, const double *x, int rows_in, int cin, int C,
                             double *a, double *s, double *y)
{
    conv_forward(n->cw[k], n->cb[k], x, rows_in, cin, C, a);
    for (int l = 0; l < rows_in / 2; l++)
        for (int co = 0; co < C; co++) {
            double t = 0.0;
            for (int ci = 0; ci < cin; ci++)
                for (int tap = 0; tap < 2; tap++)
                    t += n->pj[k][((int64_t)co * cin + ci) * 2 + tap] * x[(int64_t)(2 * l + tap) * cin + ci];
            s[(int64_t)l * C + co] = t;
        }
    for (int l = 0; l < rows_in / 2; l++)
        for (int co = 0; co < C; co++) {
            double t = n->pwb[k][co] + s[(int64_t)l * C + co];
            for (int ci = 0; ci < C; ci++) t += n->pw[k][(int64_t)co * C + ci] * a[(int64_t)l * C + ci];
            y[(int64_t)l * C + co] = t > 0.0 ? t : 0.0;
        }
}

static void cnn_forward(const oracle_cfg *c, const net_t *n, fwd_t *f)
{
    int rows = c->window, cin = NF;
    for (int k = 0; k < c->n_conv; k++) {
        if (c->residual)
            residual_forward(n, k, f->act[k], rows, cin, c->channels, f->ra, f->rs, f->act[k + 1]);
        else
            conv_forward(n->cw[k], n->cb[k], f->act[k], rows, cin, c->channels, f->act[k + 1]);
        rows /= 2;
        cin = c->channels;
    }
    /* flatten in PyTorch order: input index of (channel ch, row l) is ch * rows + l */
    const double *a = f->act[c->n_conv];
    int64_t fin = (int64_t)cin * rows;
    for (int h = 0; h < c->hidden; h++) {
        double s = n->b1[h];
        for (int ch = 0; ch < cin; ch++)
            for (int l = 0; l < rows; l++)
                s += n->w1[h * fin + (int64_t)ch * rows + l] * a[(int64_t)l * cin + ch];
        f->hid[h] = s > 0.0 ? s : 0.0;
    }
    for (int k = 0; k < n_out(c); k++) {
        double s = n->b2[k];
        for (int h = 0; h < c->hidden; h++) s += n->w2[(int64_t)k * c->hidden + h] * f->hid[h];
        f->z[k] = s;
    }
}

/* softplus(x) = log(1 + exp(x)); above 20 it returns x, as PyTorch's default threshold does */
static double softplus(double x) { return x > 20.0 ? x : log1p(exp(x)); }
static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* clamp to [0, 255], then round half to even; NaN maps to 255 */
static int to_cycles(double y)
{
    if (isnan(y)) return 255;
    if (y < 0.0) y = 0.0;
    if (y > 255.0) y = 255.0;
    return (int)nearbyint(y);
}

/* Latency t (0 fetch, 1 execution, 2 store) from the FC2 outputs z; *pre gets the
 * regression output after softplus.  Regression head: that value, clamped and
 * rounded.  Hybrid head (Sec. 2.3): the class with the largest probability,
 * i.e. the largest of the logits z[11t .. 11t+9] (softmax is monotone),
 * compared in FP64 (lowest class on exact ties); classes 0..8 are that many
 * cycles, class 9 ("more than 8") takes the regression output. */
static int head_latency(const oracle_cfg *c, const double *z, int t, double *pre)
{
    if (!c->hybrid) {
        *pre = softplus(z[t]);
        return to_cycles(*pre);
    }
    const double *lg = z + 11 * t;
    int k = 0;
    for (int j = 1; j < 10; j++)
        if (lg[j] > lg[k]) k = j;
    *pre = softplus(lg[10]);
    return k <= 8 ? k : to_cycles(*pre);
}

/* ------------------------------------------------------------------ queue + clock (Sec. 3.2) */
typedef struct {
    uint32_t rec;
    int e;              /* predicted execution latency */
    int s;              /* predicted store latency (used for stores, memory write queue only) */
    int64_t fetch_tick; /* curTick when it entered the processor queue (residence 0) */
} qent_t;

/* Ready to leave the processor queue (lat = E) or the memory write queue (lat = S). */
static int ready(const oracle_cfg *c, const qent_t *q, int lat, int64_t tick)
{
    int64_t res = tick - q->fetch_tick;
    return c->retire_strict ? (res > lat) : (res >= lat);
}

/* Processor queue: retire up to `budget` ready entries from the oldest end, in
 * order.  With the memory write queue modelled, a retired store moves to its
 * tail (keeping fetch order); other instructions leave.  Returns how many. */
static int retire_pq(const oracle_cfg *c, qent_t *q, int *len, qent_t *mq, int *mlen, int64_t tick,
                     int64_t budget)
{
    int k = 0;
    while (k < *len && k < budget && ready(c, &q[k], q[k].e, tick)) {
        if (c->store_queue && decode(q[k].rec).st) mq[(*mlen)++] = q[k];
        k++;
    }
    memmove(q, q + k, (size_t)(*len - k) * sizeof(qent_t));
    *len -= k;
    return k;
}

/* Memory write queue: retire every ready entry from the oldest end, in order,
 * with no bandwidth limit (Sec. 3.2).  Returns how many. */
static int retire_mq(const oracle_cfg *c, qent_t *mq, int *mlen, int64_t tick)
{
    int k = 0;
    while (k < *mlen && ready(c, &mq[k], mq[k].s, tick)) k++;
    memmove(mq, mq + k, (size_t)(*mlen - k) * sizeof(qent_t));
    *mlen -= k;
    return k;
}

typedef struct {
    const uint8_t *replay;   /* [n][n_lat] integer latencies to use instead of the CNN's, or NULL */
    uint8_t *lat_log;        /* [n][n_lat] latencies used */
    double *pre_log;         /* [n][n_lat] softplus outputs before clamp/round */
    int64_t *tick_log;       /* [n] curTick after the instruction's step */
    int32_t *len_log;        /* [n] processor-queue length after the step */
    int32_t *mlen_log;       /* [n] memory-write-queue length after the step */
    double *feat_log;        /* [n][W][NF] feature matrices (tiny cases only) */
    int64_t evictions, retired;
} sublog_t;

/* Simulate one sub-trace from empty queues and curTick = 0 (Sec. 3.3).
 * Returns the final curTick = sum of F + Delta (Eq. 1).
 *
 * The context of the next prediction is every instruction still in the
 * simulator, newest first: the processor queue, then the memory write queue
 * (whose stores all retired from the processor queue, so they are older).
 * Both queues together hold at most W-1 entries; appending to a full simulator
 * evicts the oldest instruction, the memory write queue's head if it has one. */
static int64_t simulate_one(const oracle_cfg *c, const net_t *net, const uint32_t *rec, int64_t n,
                            sublog_t *lg)
{
    const int W = c->window, cap = W - 1, NL = n_lat(c);
    qent_t *q = (qent_t *)malloc(sizeof(qent_t) * (size_t)(cap > 0 ? cap : 1));
    qent_t *mq = (qent_t *)malloc(sizeof(qent_t) * (size_t)(cap > 0 ? cap : 1));
    double *X = (double *)malloc(sizeof(double) * (size_t)W * NF);
    double *mem = net ? (double *)malloc(sizeof(double) * fwd_doubles(c)) : NULL;
    fwd_t f;
    int len = 0, mlen = 0;
    int64_t tick = 0;
    lg->evictions = lg->retired = 0;

    for (int64_t i = 0; i < n; i++) {
        const inst_t cur = decode(rec[i]);
        /* build the input: current instruction, then the context newest first */
        memset(X, 0, sizeof(double) * (size_t)W * NF);
        encode_static(&cur, X);
        for (int j = 1; j <= len + mlen; j++) {
            const qent_t *e = j <= len ? &q[len - j] : &mq[mlen - (j - len)];
            encode_context(&cur, e->rec, tick - e->fetch_tick, e->e, e->s, X + (size_t)j * NF);
        }
        if (lg->feat_log) memcpy(lg->feat_log + (size_t)i * W * NF, X, sizeof(double) * (size_t)W * NF);

        int L[3] = {0, 0, 0};
        if (net) {
            fwd_bind(c, mem, X, &f);
            cnn_forward(c, net, &f);
            for (int t = 0; t < NL; t++) {
                double y;
                L[t] = head_latency(c, f.z, t, &y);
                if (lg->pre_log) lg->pre_log[NL * i + t] = y;
            }
        }
        if (lg->replay)
            for (int t = 0; t < NL; t++) L[t] = lg->replay[NL * i + t];
        if (lg->lat_log)
            for (int t = 0; t < NL; t++) lg->lat_log[NL * i + t] = (uint8_t)L[t];
        const int F = L[0], E = L[1], S = L[2];

        tick += F;                                                   /* curTick += F */
        lg->retired += retire_pq(c, q, &len, mq, &mlen, tick, (int64_t)c->retire_width * F);
        if (c->store_queue) retire_mq(c, mq, &mlen, tick);
        if (len + mlen == cap) {                                     /* full: drop the oldest */
            if (mlen > 0) {
                memmove(mq, mq + 1, (size_t)(mlen - 1) * sizeof(qent_t));
                mlen--;
            } else {
                memmove(q, q + 1, (size_t)(len - 1) * sizeof(qent_t));
                len--;
            }
            lg->evictions++;
        }
        q[len].rec = rec[i];                                         /* enter with residence 0 */
        q[len].e = E;
        q[len].s = S;
        q[len].fetch_tick = tick;
        len++;
        if (lg->tick_log) lg->tick_log[i] = tick;
        if (lg->len_log) lg->len_log[i] = len;
        if (lg->mlen_log) lg->mlen_log[i] = mlen;
    }
    while (len + mlen > 0) {                                         /* drain: Delta */
        tick += 1;
        lg->retired += retire_pq(c, q, &len, mq, &mlen, tick, c->retire_width);
        if (c->store_queue) retire_mq(c, mq, &mlen, tick);
    }
    free(q);
    free(mq);
    free(X);
    free(mem);
    return tick;
}

static int cfg_ok(const oracle_cfg *c)
{
    if (c->window < 2 || c->n_conv < 1 || c->n_conv > MAXCONV) return 0;
    if ((c->window >> c->n_conv) << c->n_conv != c->window) return 0;
    if (c->channels < 1 || c->hidden < 1 || c->retire_width < 1) return 0;
    return 1;
}

int64_t oracle_blob_size(const oracle_cfg *c) { return cfg_ok(c) ? blob_size(c) : -1; }

/*
 * Simulate the listed sub-traces (all of them when `subset` is NULL).
 * Logs are indexed by global instruction position, so disjoint sub-traces
 * write disjoint parts.  With weights == NULL the CNN is skipped and `replay`
 * must give every latency (a stub predictor).  Returns 0, or -1 on bad input.
 */
int oracle_simulate(const oracle_cfg *c, const double *weights, const uint32_t *records,
                    const int64_t *offsets, int32_t n_sub, const int32_t *subset, int32_t n_subset,
                    const uint8_t *replay, int64_t *cycles_out, int64_t *evictions_out,
                    uint8_t *lat_log, double *pre_log, int64_t *tick_log, int32_t *len_log,
                    int32_t *mlen_log, double *feat_log, int32_t n_threads)
{
    if (!cfg_ok(c) || (!weights && !replay)) return -1;
    int32_t m = subset ? n_subset : n_sub;
    for (int32_t s = 0; s < m; s++) {
        int32_t b = subset ? subset[s] : s;
        if (b < 0 || b >= n_sub || offsets[b + 1] < offsets[b]) return -1;
    }
    net_t net;
    if (weights) net = net_view(c, weights);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int32_t s = 0; s < m; s++) {
        int32_t b = subset ? subset[s] : s;
        int64_t o = offsets[b], n = offsets[b + 1] - o;
        sublog_t lg;
        memset(&lg, 0, sizeof lg);
        const int NL = n_lat(c);
        lg.replay = replay ? replay + NL * o : NULL;
        lg.lat_log = lat_log ? lat_log + NL * o : NULL;
        lg.pre_log = pre_log ? pre_log + NL * o : NULL;
        lg.tick_log = tick_log ? tick_log + o : NULL;
        lg.len_log = len_log ? len_log + o : NULL;
        lg.mlen_log = mlen_log ? mlen_log + o : NULL;
        lg.feat_log = feat_log ? feat_log + o * (int64_t)c->window * NF : NULL;
        cycles_out[s] = simulate_one(c, weights ? &net : NULL, records + o, n, &lg);
        if (evictions_out) evictions_out[s] = lg.evictions;
    }
    return 0;
}

/* CNN outputs for a batch of feature matrices x [n][W][NF]: z_out [n][n_out] (FC2 outputs). */
int oracle_cnn_forward(const oracle_cfg *c, const double *weights, const double *x, int64_t n,
                       double *z_out, int32_t n_threads)
{
    if (!cfg_ok(c)) return -1;
    net_t net = net_view(c, weights);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
        double *mem = (double *)malloc(sizeof(double) * fwd_doubles(c));
        fwd_t f;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t i = 0; i < n; i++) {
            fwd_bind(c, mem, x + i * (int64_t)c->window * NF, &f);
            cnn_forward(c, &net, &f);
            for (int k = 0; k < n_out(c); k++) z_out[(int64_t)n_out(c) * i + k] = f.z[k];
        }
        free(mem);
    }
    return 0;
}

/* The latency decision of the head on given FC2 outputs z [n][n_out]: lat [n][n_lat]
 * (the integer latencies) and pre [n][n_lat] (softplus of the regression output). */
int oracle_head(const oracle_cfg *c, const double *z, int64_t n, uint8_t *lat, double *pre)
{
    if (!cfg_ok(c)) return -1;
    for (int64_t i = 0; i < n; i++)
        for (int t = 0; t < n_lat(c); t++)
            lat[n_lat(c) * i + t] = (uint8_t)head_latency(c, z + (int64_t)n_out(c) * i, t, &pre[n_lat(c) * i + t]);
    return 0;
}

/*
 * Teacher-forced training windows (labels from a timing model).  Window of
 * instruction i: row 0 = instruction i; rows 1.. = instructions i-1, i-2, ...
 * down to ctx_begin[i] (at most W-1 of them), each with residence
 * fetch[i-1] - fetch[j] and execution latency e_label[j]: the state a
 * simulator holds when it gathers instruction i, before i's fetch latency is
 * known.  x_out [n][W][NF].
 */
int oracle_window_features(const oracle_cfg *c, const uint32_t *records, int64_t n_records,
                           const int64_t *fetch, const uint8_t *e_label, const int64_t *ctx_begin,
                           const int64_t *idx, int64_t n, double *x_out)
{
    if (!cfg_ok(c)) return -1;
    const int W = c->window;
    for (int64_t s = 0; s < n; s++) {
        int64_t i = idx[s];
        if (i < 0 || i >= n_records || ctx_begin[i] < 0 || ctx_begin[i] > i) return -1;
        double *X = x_out + s * (int64_t)W * NF;
        memset(X, 0, sizeof(double) * (size_t)W * NF);
        inst_t cur = decode(records[i]);
        encode_static(&cur, X);
        int64_t now = i > 0 ? fetch[i - 1] : 0;
        for (int j = 1; j < W && i - j >= ctx_begin[i]; j++)
            encode_context(&cur, records[i - j], now - fetch[i - j], e_label[i - j], 0,
                           X + (size_t)j * NF);   /* the timing model has no write queue: S = 0 */
    }
    return 0;
}

/* ------------------------------------------------------------------ training (Sec. 2.4) */
/*
 * Loss J = mean over the n*n_lat latencies (y [n][n_lat]) of (softplus(z) - y)^2 with y the label
 * clamped to [0, 255] (squared-error loss, Sec. 2.4).  Hybrid head: the same
 * mean over the latencies of the cross-entropy of the 10 class logits against
 * class min(y, 9) plus the squared error of softplus(regression output) (the
 * paper gives no weighting; both terms count once).  grad_out gets dJ/dtheta in
 * blob order (FP64, summed over the batch in sample order).
 */
int oracle_loss_grad(const oracle_cfg *c, const double *weights, const double *x,
                     const double *y, int64_t n, double *loss_out, double *grad_out)
{
    if (!cfg_ok(c) || n <= 0 || c->residual) return -1;   /* training: plain conv layers only */
    const int W = c->window, C = c->channels, H = c->hidden, NC = c->n_conv;
    net_t net = net_view(c, weights);
    int64_t P = blob_size(c);
    memset(grad_out, 0, sizeof(double) * (size_t)P);
    net_t g = net_view(c, grad_out);   /* same offsets, into the gradient */
    double *mem = (double *)malloc(sizeof(double) * fwd_doubles(c));
    /* gradient buffers per activation */
    size_t big = (size_t)W * (NF > C ? NF : C) + (size_t)H + 16;
    double *dcur = (double *)malloc(sizeof(double) * big);
    double *dnext = (double *)malloc(sizeof(double) * big);
    double loss = 0.0;
    const int rows_n = W >> NC;
    const int64_t fin = (int64_t)C * rows_n;

    for (int64_t i = 0; i < n; i++) {
        fwd_t f;
        fwd_bind(c, mem, x + i * (int64_t)W * NF, &f);
        cnn_forward(c, &net, &f);
        double dz[MAXOUT];
        const int NL = n_lat(c);
        for (int k = 0; k < NL; k++) {
            double t = y[NL * i + k];
            t = t < 0 ? 0 : (t > 255 ? 255 : t);
            const int reg = c->hybrid ? 11 * k + 10 : k;   /* the regression output */
            double yhat = softplus(f.z[reg]);
            double r = yhat - t;
            loss += r * r;
            /* d/dz softplus(z) = sigmoid(z), and 1 above the threshold */
            double ds = f.z[reg] > 20.0 ? 1.0 : sigmoid(f.z[reg]);
            dz[reg] = 2.0 * r / ((double)NL * (double)n) * ds;
            if (c->hybrid) {
                /* cross-entropy: log-sum-exp of the logits minus the target class's */
                const double *lg = f.z + 11 * k;
                const int cls = t > 8.0 ? 9 : (int)t;
                double mx = lg[0];
                for (int j = 1; j < 10; j++) mx = lg[j] > mx ? lg[j] : mx;
                double se = 0.0;
                for (int j = 0; j < 10; j++) se += exp(lg[j] - mx);
                loss += mx + log(se) - lg[cls];
                for (int j = 0; j < 10; j++)
                    dz[11 * k + j] = (exp(lg[j] - mx) / se - (j == cls ? 1.0 : 0.0)) / ((double)NL * (double)n);
            }
        }
        /* FC2 */
        double *dh = dcur;
        for (int h = 0; h < H; h++) dh[h] = 0.0;
        for (int k = 0; k < n_out(c); k++) {
            ((double *)g.b2)[k] += dz[k];
            for (int h = 0; h < H; h++) {
                ((double *)g.w2)[(int64_t)k * H + h] += dz[k] * f.hid[h];
                dh[h] += dz[k] * net.w2[(int64_t)k * H + h];
            }
        }
        /* ReLU of FC1 */
        for (int h = 0; h < H; h++) if (f.hid[h] <= 0.0) dh[h] = 0.0;
        /* FC1 over the PyTorch-order flatten */
        const double *a = f.act[NC];
        double *da = dnext;
        for (int64_t q = 0; q < (int64_t)rows_n * C; q++) da[q] = 0.0;
        for (int h = 0; h < H; h++) {
            ((double *)g.b1)[h] += dh[h];
            for (int ch = 0; ch < C; ch++)
                for (int l = 0; l < rows_n; l++) {
                    ((double *)g.w1)[h * fin + (int64_t)ch * rows_n + l] += dh[h] * a[(int64_t)l * C + ch];
                    da[(int64_t)l * C + ch] += dh[h] * net.w1[h * fin + (int64_t)ch * rows_n + l];
                }
        }
        /* conv layers, last to first */
        for (int k = NC - 1; k >= 0; k--) {
            int rows_out = W >> (k + 1), rows_in = W >> k;
            int cin = k == 0 ? NF : C;
            const double *yk = f.act[k + 1], *xk = f.act[k];
            double *dy = da;                       /* [rows_out][C] */
            for (int64_t q = 0; q < (int64_t)rows_out * C; q++) if (yk[q] <= 0.0) dy[q] = 0.0;
            double *dx = (da == dnext) ? dcur : dnext;  /* [rows_in][cin] */
            for (int64_t q = 0; q < (int64_t)rows_in * cin; q++) dx[q] = 0.0;
            for (int l = 0; l < rows_out; l++)
                for (int co = 0; co < C; co++) {
                    double d = dy[(int64_t)l * C + co];
                    if (d == 0.0) continue;
                    ((double *)g.cb[k])[co] += d;
                    for (int ci = 0; ci < cin; ci++)
                        for (int t = 0; t < 2; t++) {
                            int64_t wi = ((int64_t)co * cin + ci) * 2 + t;
                            ((double *)g.cw[k])[wi] += d * xk[(int64_t)(2 * l + t) * cin + ci];
                            dx[(int64_t)(2 * l + t) * cin + ci] += d * net.cw[k][wi];
                        }
                }
            da = dx;
        }
    }
    *loss_out = loss / ((double)n_lat(c) * (double)n);
    free(mem);
    free(dcur);
    free(dnext);
    return 0;
}

/* One Adam step (Kingma & Ba; beta1, beta2, eps as given, no weight decay), step t >= 1. */
void oracle_adam(double *theta, double *m, double *v, const double *g, int64_t n, double lr,
                 double beta1, double beta2, double eps, int64_t t)
{
    double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t i = 0; i < n; i++) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        theta[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
