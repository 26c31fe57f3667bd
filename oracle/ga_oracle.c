/*
 * ga_oracle.c -- plain, slow CPU oracle for the synchronous trackable island-model GA.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls this
 * file; only the tests, the package's smoke check and the benchmark's CPU-baseline leg
 * do.  It shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (Moreno et al., "Trackable Island-model Genetic Algorithms at Wafer
 * Scale", GECCO'24 Companion):
 *   - Sec. 2: every island hosts an independent population and trades genomes with its
 *     four cardinal neighbours; each generation handles migration first, then evaluation,
 *     tournament selection (n random picks, ties broken randomly), mutation of the whole
 *     next population and an hstrat annotation update for the elapsed generation; the run
 *     halts at a generation count.
 *   - Sec. 3: tournament size 5, 32 genomes per island, purifying-only vs adaptive
 *     treatments.
 *   - Fig. 1 caption: hstrat markers allow post hoc estimates of relatedness; here that is
 *     the pairwise MRCA-bound computation.
 * Where the paper is silent (curation rule, draw schedule, tie-break, torus edges) the
 * readings below are this project's and are listed, with reasons, in the design notes.
 *
 * The data layout here is structure-of-arrays (trait[], counter[], surface[][]); only
 * orc_snapshot writes the library's canonical agent record.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------ */
/* Counter-based random numbers: Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw,  */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).  One round maps the counter     */
/* (c0,c1,c2,c3) with key (k0,k1) to (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1,      */
/* lo(M0*c0)); the key is advanced by the Weyl constants between rounds.                  */
/* ------------------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t x[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k[2] = {key_in[0], key_in[1]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k[0] += PHILOX_W0;
            k[1] += PHILOX_W1;
        }
        uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)x[0];
        uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)x[2];
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y[4];
        y[0] = hi1 ^ x[1] ^ k[0];
        y[1] = lo1;
        y[2] = hi0 ^ x[3] ^ k[1];
        y[3] = lo0;
        memcpy(x, y, sizeof x);
    }
    memcpy(out, x, sizeof x);
}

/* Draw purposes: the third counter word is (slot | purpose << 16). */
#define ORC_PURPOSE_BIRTH   1u
#define ORC_PURPOSE_FOUNDER 2u
#define ORC_PURPOSE_MUTATE  3u

static void draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t slot, uint32_t purpose,
                 uint32_t run_id, uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, slot | (purpose << 16), run_id};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------------------ */
/* Normal deviates for the float-fitness treatments of Sec. 3 ("decreased / increased     */
/* fitness by a normally-distributed amount"), by the Box-Muller transform,               */
/* z = sqrt(-2 ln u1) cos(2 pi u2), in IEEE single precision from correctly rounded       */
/* operations only (+, -, *, /, sqrt; this file is compiled without FMA contraction), so   */
/* that any other implementation performing the same operations gets the same bits:       */
/*   ln x, x in (0, 1]: x = m 2^e with m in [0.5, 1) read from the float's bits;          */
/*     ln m = 2 atanh(s), s = (m - 1)/(m + 1), by the series 2 s (1 + s^2/3 + ... + s^12/13) */
/*     in Horner form; ln x = e ln 2 + ln m.                                               */
/*   cos(2 pi k / 2^24): quadrant q = k >> 22, angle a = (k mod 2^22) 2^-22 (pi/2); the     */
/*     Taylor series of cos a (to a^14) and sin a (to a^15) in Horner form, then           */
/*     cos, -sin, -cos, sin for q = 0, 1, 2, 3.                                             */
/*   u1 = (k1 + 1) 2^-24 in (0, 1], k1 = top 24 bits of word a; k = top 24 bits of word b. */
/* ------------------------------------------------------------------------------------ */
static float unit_log(float x)
{
    uint32_t bits;
    memcpy(&bits, &x, 4);
    const int e = (int)((bits >> 23) & 0xFFu) - 126;
    const uint32_t mbits = (bits & 0x007FFFFFu) | 0x3F000000u;
    float m;
    memcpy(&m, &mbits, 4);
    const float s = (m - 1.0f) / (m + 1.0f);
    const float t = s * s;
    float p = (float)(1.0 / 13.0);
    p = p * t + (float)(1.0 / 11.0);
    p = p * t + (float)(1.0 / 9.0);
    p = p * t + (float)(1.0 / 7.0);
    p = p * t + (float)(1.0 / 5.0);
    p = p * t + (float)(1.0 / 3.0);
    p = p * t + 1.0f;
    const float ln_m = (2.0f * s) * p;
    return (float)e * (float)0.69314718055994530942 + ln_m;
}

static float turn_cos(uint32_t k)
{
    const uint32_t q = (k >> 22) & 3u;
    const float a = ((float)(k & 0x3FFFFFu) * (float)(1.0 / 4194304.0)) *
                    (float)(3.14159265358979323846 / 2.0);
    const float a2 = a * a;
    float c = -(float)(1.0 / 87178291200.0); /* -1/14! */
    c = c * a2 + (float)(1.0 / 479001600.0); /*  1/12! */
    c = c * a2 - (float)(1.0 / 3628800.0);   /* -1/10! */
    c = c * a2 + (float)(1.0 / 40320.0);     /*  1/8!  */
    c = c * a2 - (float)(1.0 / 720.0);       /* -1/6!  */
    c = c * a2 + (float)(1.0 / 24.0);        /*  1/4!  */
    c = c * a2 - 0.5f;                       /* -1/2!  */
    c = c * a2 + 1.0f;
    float sn = -(float)(1.0 / 1307674368000.0); /* -1/15! */
    sn = sn * a2 + (float)(1.0 / 6227020800.0); /*  1/13! */
    sn = sn * a2 - (float)(1.0 / 39916800.0);   /* -1/11! */
    sn = sn * a2 + (float)(1.0 / 362880.0);     /*  1/9!  */
    sn = sn * a2 - (float)(1.0 / 5040.0);       /* -1/7!  */
    sn = sn * a2 + (float)(1.0 / 120.0);        /*  1/5!  */
    sn = sn * a2 - (float)(1.0 / 6.0);          /* -1/3!  */
    sn = sn * a2 + 1.0f;
    sn = sn * a;
    switch (q) {
    case 0: return c;
    case 1: return -sn;
    case 2: return -c;
    default: return sn;
    }
}

float orc_unit_log(float x) { return unit_log(x); }
float orc_turn_cos(uint32_t k) { return turn_cos(k); }

float orc_normal(uint32_t a, uint32_t b)
{
    const float u1 = (float)((a >> 8) + 1u) * (float)(1.0 / 16777216.0);
    const float r = sqrtf(-2.0f * unit_log(u1));
    return r * turn_cos(b >> 8);
}

/* ------------------------------------------------------------------------------------ */
/* Hereditary-stratigraphy curation: which surface site the deposit of rank T overwrites. */
/* The paper only says the annotations are "updated to reflect an elapsed generation"     */
/* (Sec. 2); the policies below are this project's readings.  -1 means "not stored".      */
/* ------------------------------------------------------------------------------------ */
enum { ORC_STEADY = 0, ORC_TILTED = 1, ORC_HYBRID = 2 };

static uint32_t bit_length(uint64_t x)
{
    uint32_t n = 0;
    while (x) {
        ++n;
        x >>= 1;
    }
    return n;
}

/* hanoi value of rank T: the number of times 2 divides T + 1 */
static uint32_t hanoi_value(uint64_t T)
{
    uint64_t u = T + 1;
    uint32_t h = 0;
    while ((u & 1u) == 0) {
        ++h;
        u >>= 1;
    }
    return h;
}

static uint32_t exact_log2(uint32_t v)
{
    uint32_t s = 0;
    while ((1u << s) < v) ++s;
    return s;
}

/*
 * Steady curation over S = 2^s sites.  Ranks 0..S-1 fill the sites in order.  Epoch t >= 1
 * covers T in [2^(s+t-1), 2^(s+t)).  During epoch t a rank is kept iff its hanoi value is
 * at least t, and each kept rank takes over the site of the OLDEST still-retained rank whose
 * hanoi value is exactly t-1.  At the end of epoch t the retained ranks are therefore
 * exactly { r < 2^(s+t) : hanoi(r) >= t }, evenly spaced 2^t apart.
 */
int64_t orc_site_steady(uint32_t S, uint64_t T)
{
    uint32_t s = exact_log2(S);
    if (T < S) return (int64_t)T;
    uint32_t t = bit_length(T) - s;
    if (hanoi_value(T) < t) return -1;
    /* kept ranks of epoch t are T+1 = m*2^t with m in (S/2, S]; the j-th of them (j = 0,1,..)
       replaces the j-th rank with hanoi value exactly t-1, i.e. (2j+1)*2^(t-1) - 1 */
    uint64_t j = ((T + 1) >> t) - (S / 2) - 1;
    uint64_t victim = ((2 * j + 1) << (t - 1)) - 1;
    return orc_site_steady(S, victim);
}

/*
 * Tilted (recency-weighted) curation over S sites, S even: the sites form L = S/2 levels
 * of two sites each.  Level h < L-1 keeps the two most recent ranks whose hanoi value is
 * exactly h; the top level keeps the two most recent ranks with hanoi value >= L-1.
 * Ranks of one class alternate between the two sites of their level (a ring of two).
 */
int64_t orc_site_tilted(uint32_t S, uint64_t T)
{
    uint32_t L = S / 2;
    uint32_t h = hanoi_value(T);
    uint64_t earlier; /* ranks below T in the same class */
    uint32_t level;
    if (h < L - 1) {
        level = h;
        earlier = T >> (h + 1); /* T + 1 = (2q+1) 2^h  =>  q = floor(T / 2^(h+1)) */
    } else {
        level = L - 1;
        earlier = ((T + 1) >> (L - 1)) - 1; /* T + 1 = q' 2^(L-1), q' = 1, 2, ... */
    }
    return (int64_t)(2u * level + (uint32_t)(earlier & 1u));
}

/* Hybrid: the first S/2 sites run steady on even ranks, the last S/2 run tilted on odd ranks. */
int64_t orc_site_hybrid(uint32_t S, uint64_t T)
{
    if ((T & 1u) == 0) return orc_site_steady(S / 2, T / 2);
    return (int64_t)(S / 2) + orc_site_tilted(S / 2, (T - 1) / 2);
}

int64_t orc_site(uint32_t policy, uint32_t S, uint64_t T)
{
    switch (policy) {
    case ORC_STEADY: return orc_site_steady(S, T);
    case ORC_TILTED: return orc_site_tilted(S, T);
    case ORC_HYBRID: return orc_site_hybrid(S, T);
    default: return -2;
    }
}

/* Sites of ranks t0 .. t0 + count - 1, one call of orc_site each. */
void orc_site_table(uint32_t policy, uint32_t S, uint64_t t0, uint64_t count, int64_t *out)
{
    for (uint64_t i = 0; i < count; ++i) out[i] = orc_site(policy, S, t0 + i);
}

/* ------------------------------------------------------------------------------------ */
/* The synchronous island GA.                                                            */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    uint32_t rows, cols;        /* torus of islands, island id = y * cols + x           */
    uint32_t island_size;       /* N, a power of two in [4, 256]                         */
    uint32_t tournament_size;   /* n in [1, 8]                                           */
    double p_ben, p_del;        /* per-birth probabilities of a +1 / -1 trait mutation   */
    uint32_t surface_sites;     /* S                                                     */
    uint32_t differentia_bits;  /* b in {1, 2, 4, 8}                                     */
    uint32_t curation;          /* ORC_STEADY / ORC_TILTED / ORC_HYBRID                  */
    uint32_t migrate_every;     /* k: migrate when g mod k == 0; 0 disables migration    */
    uint64_t seed;
    uint32_t run_id;
    uint32_t threads;           /* worker threads for the per-island loops (0 or 1: one) */
    uint32_t model;             /* ORC_MODEL_TRAIT or ORC_MODEL_FITNESS                  */
    double effect_scale;        /* ORC_MODEL_FITNESS: mutation amount = scale * |z|      */
} orc_config;

/* Genome models.  TRAIT: int32 trait, +1 / -1 mutations.  FITNESS (Sec. 3 treatments): the
   first word is an IEEE float fitness; a deleterious mutation subtracts, a beneficial one
   adds, effect_scale * |z| with z a standard normal deviate drawn from
   Philox((g, island, slot | MUTATE << 16, run)) words 0 and 1. */
enum { ORC_MODEL_TRAIT = 0, ORC_MODEL_FITNESS = 1 };

typedef struct {
    orc_config cfg;
    uint32_t n_islands, n_agents, words; /* words = surface words per agent */
    uint32_t theta_ben, theta_del;
    uint64_t gen;                        /* generations elapsed */
    int32_t *trait;
    uint32_t *counter;
    uint32_t *surface;                   /* n_agents * words */
    /* scratch for one generation */
    int32_t *trait2;
    uint32_t *counter2;
    uint32_t *surface2;
    /* asynchronous mode: per island and direction, the send buffer towards that neighbour
       (state and one agent); allocated on first use, all zero = every buffer empty */
    uint32_t *mail_full;  /* 0: empty, 1: full */
    int32_t *mail_trait;
    uint32_t *mail_counter;
    uint32_t *mail_surface;
    /* lineage tracking (tests only; off unless orc_track_lineage was called): every agent
       carries the id of the birth that made it, g * n_agents + slot (-1: founder); event_parent
       maps a birth to its parent's birth, event_depth to the child's counter */
    int64_t *tag, *tag2, *mail_tag;
    int64_t *event_parent;
    uint32_t *event_depth;
    uint64_t event_cap;   /* generations covered by the event arrays */
} orc_state;

/* probability -> 32-bit threshold, once, in IEEE double: theta = min(2^32-1, floor(p 2^32)) */
static uint32_t threshold(double p)
{
    double x = floor(p * 4294967296.0);
    if (x < 0.0) x = 0.0;
    if (x > 4294967295.0) x = 4294967295.0;
    return (uint32_t)x;
}

static int is_pow2(uint32_t v) { return v && !(v & (v - 1)); }

int orc_validate(const orc_config *c)
{
    if (!c) return -1;
    if (c->rows == 0 || c->cols == 0) return -1;
    if (!is_pow2(c->island_size) || c->island_size < 4 || c->island_size > 256) return -1;
    if (c->tournament_size < 1 || c->tournament_size > 8) return -1;
    if (!(c->p_ben >= 0.0) || !(c->p_del >= 0.0) || c->p_ben + c->p_del > 1.0) return -1;
    if (!(c->differentia_bits == 1 || c->differentia_bits == 2 || c->differentia_bits == 4 ||
          c->differentia_bits == 8))
        return -1;
    if (!is_pow2(c->surface_sites)) return -1;
    if (c->curation == ORC_STEADY && c->surface_sites < 4) return -1;
    if (c->curation == ORC_TILTED && c->surface_sites < 4) return -1;
    if (c->curation == ORC_HYBRID && c->surface_sites < 8) return -1;
    if (c->curation > ORC_HYBRID) return -1;
    if ((uint64_t)c->surface_sites * c->differentia_bits > 256) return -1;
    if ((uint64_t)c->rows * c->cols * c->island_size > 0xFFFFFFFFull) return -1;
    if (c->model > ORC_MODEL_FITNESS) return -1;
    if (c->model == ORC_MODEL_FITNESS && !(c->effect_scale > 0.0 && c->effect_scale < 1e30))
        return -1;
    return 0;
}

void orc_destroy(orc_state *st)
{
    if (!st) return;
    free(st->trait);
    free(st->counter);
    free(st->surface);
    free(st->trait2);
    free(st->counter2);
    free(st->surface2);
    free(st->mail_full);
    free(st->mail_trait);
    free(st->mail_counter);
    free(st->mail_surface);
    free(st->tag);
    free(st->tag2);
    free(st->mail_tag);
    free(st->event_parent);
    free(st->event_depth);
    free(st);
}

/* Founder (Sec. 2 "initialize"): every agent is a clone of one founder with trait 0,
   counter 0, and surface word w drawn as word 0 of Philox((0, 0, w | FOUNDER << 16, run)). */
orc_state *orc_create(const orc_config *cfg)
{
    if (orc_validate(cfg) != 0) return NULL;
    orc_state *st = (orc_state *)calloc(1, sizeof *st);
    if (!st) return NULL;
    st->cfg = *cfg;
    st->n_islands = cfg->rows * cfg->cols;
    st->n_agents = st->n_islands * cfg->island_size;
    st->words = (cfg->surface_sites * cfg->differentia_bits + 31) / 32;
    st->theta_ben = threshold(cfg->p_ben);
    st->theta_del = threshold(cfg->p_del);
    size_t n = st->n_agents;
    st->trait = (int32_t *)calloc(n, sizeof(int32_t));
    st->counter = (uint32_t *)calloc(n, sizeof(uint32_t));
    st->surface = (uint32_t *)calloc(n * st->words, sizeof(uint32_t));
    st->trait2 = (int32_t *)calloc(n, sizeof(int32_t));
    st->counter2 = (uint32_t *)calloc(n, sizeof(uint32_t));
    st->surface2 = (uint32_t *)calloc(n * st->words, sizeof(uint32_t));
    if (!st->trait || !st->counter || !st->surface || !st->trait2 || !st->counter2 ||
        !st->surface2) {
        orc_destroy(st);
        return NULL;
    }
    uint32_t founder[8] = {0};
    for (uint32_t w = 0; w < st->words; ++w) {
        uint32_t r[4];
        draw(cfg->seed, 0, 0, w, ORC_PURPOSE_FOUNDER, cfg->run_id, r);
        founder[w] = r[0];
    }
    /* bits past S*b in the top word are not part of the surface: they are kept at zero */
    uint32_t used = (cfg->surface_sites * cfg->differentia_bits) % 32;
    if (used) founder[st->words - 1] &= (1u << used) - 1u;
    for (size_t a = 0; a < n; ++a)
        for (uint32_t w = 0; w < st->words; ++w) st->surface[a * st->words + w] = founder[w];
    return st;
}

uint64_t orc_generation(const orc_state *st) { return st->gen; }
uint32_t orc_agent_count(const orc_state *st) { return st->n_agents; }

static int worker_threads(const orc_state *st)
{
    return st->cfg.threads > 1 ? (int)st->cfg.threads : 1;
}

/* torus neighbour of island `isl` in direction d: 0 north (y-1), 1 south (y+1),
   2 east (x+1), 3 west (x-1) */
static uint32_t neighbour(const orc_config *c, uint32_t isl, int d)
{
    uint32_t y = isl / c->cols, x = isl % c->cols;
    switch (d) {
    case 0: y = (y + c->rows - 1) % c->rows; break;
    case 1: y = (y + 1) % c->rows; break;
    case 2: x = (x + 1) % c->cols; break;
    default: x = (x + c->cols - 1) % c->cols; break;
    }
    return y * c->cols + x;
}

static void copy_agent(orc_state *st, int32_t *t_dst, uint32_t *c_dst, uint32_t *s_dst,
                       uint32_t dst, const int32_t *t_src, const uint32_t *c_src,
                       const uint32_t *s_src, uint32_t src)
{
    t_dst[dst] = t_src[src];
    c_dst[dst] = c_src[src];
    memcpy(&s_dst[(size_t)dst * st->words], &s_src[(size_t)src * st->words],
           st->words * sizeof(uint32_t));
}

/* Lineage tags follow genomes: a copy keeps the tag, a birth gets a new one. */
static int tracking(const orc_state *st) { return st->tag != NULL; }

static void record_birth(orc_state *st, uint32_t g, uint32_t child, uint32_t parent)
{
    const uint64_t id = (uint64_t)g * st->n_agents + child;
    st->event_parent[id] = st->tag[parent];
    st->event_depth[id] = st->counter2[child] + 1u; /* the child's counter after the birth */
    st->tag2[child] = (int64_t)id;
}

/* Make room for birth records of generations below `gen_end`. */
static int reserve_events(orc_state *st, uint64_t gen_end)
{
    if (!tracking(st) || gen_end <= st->event_cap) return 0;
    uint64_t cap = st->event_cap ? st->event_cap : 64;
    while (cap < gen_end) cap *= 2;
    const size_t n = (size_t)(cap * st->n_agents);
    int64_t *p = (int64_t *)realloc(st->event_parent, n * sizeof(int64_t));
    if (!p) return -2;
    st->event_parent = p;
    uint32_t *d = (uint32_t *)realloc(st->event_depth, n * sizeof(uint32_t));
    if (!d) return -2;
    st->event_depth = d;
    st->event_cap = cap;
    return 0;
}

/*
 * Migration of generation g (Sec. 2: handled first; each island receives genomes from its
 * four cardinal neighbours, which replace randomly chosen members).  Reading used here:
 *   - one migrant per direction per migration generation, on a torus;
 *   - the migrant from neighbour nb(d) is a uniform random member (a copy) of nb(d)'s
 *     population as it stood before any migrant of this generation landed;
 *   - the random words come from the receiving island's own birth draws of generation g:
 *     for direction d, word 3 of the draw of slot d supplies the migrant index
 *     e = (bits 8..15) * N >> 8 and the placement r = d + (bits 16..31) * (N - d) >> 16;
 *   - the four arrivals land in four distinct slots chosen by a partial Fisher-Yates
 *     shuffle in direction order N, S, E, W.
 * src_ids (optional, n_agents) receives, for every slot, the id of the pre-migration agent
 * whose genome it now holds.
 */
void orc_migrate(orc_state *st, uint32_t *src_ids)
{
    const orc_config *c = &st->cfg;
    const uint32_t N = c->island_size;
    const uint32_t g = (uint32_t)st->gen;
    /* snapshot of the pre-migration population */
    memcpy(st->trait2, st->trait, st->n_agents * sizeof(int32_t));
    memcpy(st->counter2, st->counter, st->n_agents * sizeof(uint32_t));
    memcpy(st->surface2, st->surface, (size_t)st->n_agents * st->words * sizeof(uint32_t));
    if (tracking(st)) memcpy(st->tag2, st->tag, st->n_agents * sizeof(int64_t));
    if (src_ids)
        for (uint32_t a = 0; a < st->n_agents; ++a) src_ids[a] = a;

#pragma omp parallel for schedule(static) num_threads(worker_threads(st))
    for (int64_t isl64 = 0; isl64 < (int64_t)st->n_islands; ++isl64) {
        uint32_t isl = (uint32_t)isl64;
        uint32_t perm[256];
        for (uint32_t j = 0; j < N; ++j) perm[j] = j;
        for (uint32_t d = 0; d < 4; ++d) {
            uint32_t w[4];
            draw(c->seed, g, isl, d, ORC_PURPOSE_BIRTH, c->run_id, w);
            uint32_t e = (((w[3] >> 8) & 0xFFu) * N) >> 8;
            uint32_t r = d + (uint32_t)((((uint64_t)(w[3] >> 16)) * (N - d)) >> 16);
            uint32_t tmp = perm[d];
            perm[d] = perm[r];
            perm[r] = tmp;
            uint32_t dst = isl * N + perm[d];
            uint32_t src = neighbour(c, isl, (int)d) * N + e;
            copy_agent(st, st->trait, st->counter, st->surface, dst, st->trait2, st->counter2,
                       st->surface2, src);
            if (tracking(st)) st->tag[dst] = st->tag2[src];
            if (src_ids) src_ids[dst] = src;
        }
    }
}

/*
 * Evaluation, tournament selection, copy, mutation and hstrat deposit of generation g
 * (Sec. 2, in that order), then g += 1.
 *   - fitness = trait;
 *   - child slot j draws Philox((g, island, j | BIRTH << 16, run)) = (B0, B1, B2, B3);
 *     tournament draw i (i < n) is idx_i = byte_(i mod 4)(i < 4 ? B0 : B1) * N >> 8, with
 *     replacement; the parent is the candidate of largest trait, the earliest draw winning
 *     ties (draw order is itself uniform, so this is a random tie-break);
 *   - child = copy of the parent; with x = B2: x < theta_del => trait -= 1, otherwise
 *     x - theta_del < theta_ben => trait += 1 (32-bit two's-complement arithmetic);
 *   - hstrat: site = curation(S, c) for the child's inherited counter c; when stored, the
 *     low b bits of B3 overwrite bits [site*b, site*b + b) of the surface; then c += 1.
 * parent_slots (optional, n_agents) receives the winning slot index of every child.
 */
static void reproduce_island(orc_state *st, uint32_t isl, uint32_t g, uint32_t *parent_slots)
{
    const orc_config *c = &st->cfg;
    const uint32_t N = c->island_size, n = c->tournament_size, b = c->differentia_bits;
    const uint32_t words = st->words;
    const uint32_t base = isl * N;
    for (uint32_t j = 0; j < N; ++j) {
        uint32_t w[4];
        draw(c->seed, g, isl, j, ORC_PURPOSE_BIRTH, c->run_id, w);
        /* tournament */
        uint32_t best = 0;
        for (uint32_t i = 0; i < n; ++i) {
            uint32_t word = i < 4 ? w[0] : w[1];
            uint32_t byte = (word >> (8 * (i % 4))) & 0xFFu;
            uint32_t idx = (byte * N) >> 8;
            int better;
            if (c->model == ORC_MODEL_FITNESS) {
                float fi, fb;
                memcpy(&fi, &st->trait[base + idx], 4);
                memcpy(&fb, &st->trait[base + best], 4);
                better = fi > fb;
            } else {
                better = st->trait[base + idx] > st->trait[base + best];
            }
            if (i == 0 || better) best = idx;
        }
        if (parent_slots) parent_slots[base + j] = best;
        /* copy */
        uint32_t child = base + j, parent = base + best;
        copy_agent(st, st->trait2, st->counter2, st->surface2, child, st->trait,
                   st->counter, st->surface, parent);
        if (tracking(st)) record_birth(st, g, child, parent);
        /* mutate */
        uint32_t x = w[2];
        int del = x < st->theta_del;
        int ben = !del && x - st->theta_del < st->theta_ben;
        if (c->model == ORC_MODEL_FITNESS) {
            if (del || ben) {
                uint32_t mw[4];
                draw(c->seed, g, isl, j, ORC_PURPOSE_MUTATE, c->run_id, mw);
                const float amount = (float)c->effect_scale * fabsf(orc_normal(mw[0], mw[1]));
                float f;
                memcpy(&f, &st->trait2[child], 4);
                f = del ? f - amount : f + amount;
                memcpy(&st->trait2[child], &f, 4);
            }
        } else if (del) {
            st->trait2[child] = (int32_t)((uint32_t)st->trait2[child] - 1u);
        } else if (ben) {
            st->trait2[child] = (int32_t)((uint32_t)st->trait2[child] + 1u);
        }
        /* hstrat deposit for the elapsed generation */
        int64_t site = orc_site(c->curation, c->surface_sites, st->counter2[child]);
        if (site >= 0) {
            uint32_t pos = (uint32_t)site * b;
            uint32_t *sw = &st->surface2[(size_t)child * words + pos / 32];
            uint32_t mask = (b == 32 ? 0xFFFFFFFFu : ((1u << b) - 1u)) << (pos % 32);
            *sw = (*sw & ~mask) | ((w[3] << (pos % 32)) & mask);
        }
        st->counter2[child] += 1u;
    }
}

/* One generation of every island (each reads only its own members), then g += 1. */
void orc_reproduce(orc_state *st, uint32_t *parent_slots)
{
    const uint32_t g = (uint32_t)st->gen;
    if (reserve_events(st, st->gen + 1) != 0) abort();
#pragma omp parallel for schedule(static) num_threads(worker_threads(st))
    for (int64_t isl64 = 0; isl64 < (int64_t)st->n_islands; ++isl64)
        reproduce_island(st, (uint32_t)isl64, g, parent_slots);
    /* the next population replaces the current one */
    int32_t *tt = st->trait;
    st->trait = st->trait2;
    st->trait2 = tt;
    uint32_t *cc = st->counter;
    st->counter = st->counter2;
    st->counter2 = cc;
    uint32_t *ss = st->surface;
    st->surface = st->surface2;
    st->surface2 = ss;
    int64_t *gg = st->tag;
    st->tag = st->tag2;
    st->tag2 = gg;
    st->gen += 1;
}

/* One full generation: migration when due, then reproduction. */
void orc_step(orc_state *st, uint32_t n_gens)
{
    for (uint32_t i = 0; i < n_gens; ++i) {
        uint32_t k = st->cfg.migrate_every;
        if (k != 0 && st->gen % k == 0) orc_migrate(st, NULL);
        orc_reproduce(st, NULL);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Asynchronous migration (Sec. 2: the wafer-scale loop posts and collects migrants       */
/* without waiting), on the sequential schedule: within a window of generations the       */
/* islands run one after another in index order, each through all of the window.          */
/* ------------------------------------------------------------------------------------ */

static int async_alloc(orc_state *st)
{
    if (st->mail_full) return 0;
    const size_t boxes = (size_t)st->n_islands * 4;
    st->mail_full = (uint32_t *)calloc(boxes, sizeof(uint32_t));
    st->mail_trait = (int32_t *)calloc(boxes, sizeof(int32_t));
    st->mail_counter = (uint32_t *)calloc(boxes, sizeof(uint32_t));
    st->mail_surface = (uint32_t *)calloc(boxes * st->words, sizeof(uint32_t));
    if (!st->mail_full || !st->mail_trait || !st->mail_counter || !st->mail_surface) return -2;
    return 0;
}

static void async_clear(orc_state *st)
{
    if (!st->mail_full) return;
    const size_t boxes = (size_t)st->n_islands * 4;
    memset(st->mail_full, 0, boxes * sizeof(uint32_t));
    memset(st->mail_trait, 0, boxes * sizeof(int32_t));
    memset(st->mail_counter, 0, boxes * sizeof(uint32_t));
    memset(st->mail_surface, 0, boxes * st->words * sizeof(uint32_t));
}

/*
 * Migration step of island `isl` at its generation g (Sec. 2: the update loop first tests
 * every completion flag; then, for each receive that completed, the arrived genome replaces
 * a randomly chosen member; then, for each send that completed, the send buffer is refilled
 * with a randomly sampled member; only after that are flags reset and new sends started).
 * Reading used here: each island has one send buffer per direction holding at most one
 * genome; a send completes when the neighbour takes the genome out.
 *   1. test: R_d = the buffer of neighbour nb(d) facing isl (nb(d)'s direction opposite to
 *      d) is full; E_d = isl's own buffer towards d is empty -- all eight tested first;
 *   2. collect: for d = N, S, E, W in order, the partial Fisher-Yates draw of the synchronous
 *      mode swaps position d with r_d (whether or not anything arrives); if R_d, the genome
 *      is taken out of the buffer (which becomes empty) and replaces the member in position d;
 *   3. refill: for each d with E_d, a copy of member e_d = (bits 8..15 of word 3 of slot d's
 *      draw) * N >> 8 of the island as it stands after step 2 fills isl's buffer towards d.
 * The flags are only ever changed by the island that owns a buffer (fill) and by the one
 * that takes from it, so testing them first differs from testing each one when it is used
 * only where an island is its own neighbour (one-row or one-column tori): a buffer that the
 * island empties itself in step 2 was full when tested and is refilled a pass later.
 * arrivals (optional, 4 per island) counts deliveries per direction.
 */
static void async_migrate_island(orc_state *st, uint32_t isl, uint32_t g, uint64_t *arrivals)
{
    const orc_config *c = &st->cfg;
    const uint32_t N = c->island_size, words = st->words;
    uint32_t w3[4], in_box[4];
    int full_in[4], empty_out[4];
    for (uint32_t d = 0; d < 4; ++d) {
        uint32_t w[4];
        draw(c->seed, g, isl, d, ORC_PURPOSE_BIRTH, c->run_id, w);
        w3[d] = w[3];
        in_box[d] = neighbour(c, isl, (int)d) * 4 + (d ^ 1u);
        full_in[d] = st->mail_full[in_box[d]] != 0;
        empty_out[d] = st->mail_full[isl * 4 + d] == 0;
    }
    uint32_t perm[256];
    for (uint32_t j = 0; j < N; ++j) perm[j] = j;
    for (uint32_t d = 0; d < 4; ++d) {
        uint32_t r = d + (uint32_t)((((uint64_t)(w3[d] >> 16)) * (N - d)) >> 16);
        uint32_t tmp = perm[d];
        perm[d] = perm[r];
        perm[r] = tmp;
        if (!full_in[d]) continue;
        const uint32_t box = in_box[d], dst = isl * N + perm[d];
        st->trait[dst] = st->mail_trait[box];
        st->counter[dst] = st->mail_counter[box];
        memcpy(&st->surface[(size_t)dst * words], &st->mail_surface[(size_t)box * words],
               words * sizeof(uint32_t));
        if (tracking(st)) st->tag[dst] = st->mail_tag[box];
        st->mail_full[box] = 0;
        if (arrivals) arrivals[isl * 4 + d] += 1;
    }
    for (uint32_t d = 0; d < 4; ++d) {
        if (!empty_out[d]) continue;
        const uint32_t e = (((w3[d] >> 8) & 0xFFu) * N) >> 8;
        const uint32_t src = isl * N + e, box = isl * 4 + d;
        st->mail_trait[box] = st->trait[src];
        st->mail_counter[box] = st->counter[src];
        memcpy(&st->mail_surface[(size_t)box * words], &st->surface[(size_t)src * words],
               words * sizeof(uint32_t));
        if (tracking(st)) st->mail_tag[box] = st->tag[src];
        st->mail_full[box] = 1;
    }
}

/*
 * One window of n_gens generations on the sequential schedule: for each island in index
 * order, generations gen .. gen + n_gens - 1 (the migration step above when the migration
 * policy says so, then evaluation, selection, mutation and deposit -- the deposit site
 * follows the agent's own counter); then gen += n_gens.  arrivals as above.
 * Returns 0, or -2 when out of memory.
 */
int orc_step_async(orc_state *st, uint32_t n_gens, uint64_t *arrivals)
{
    if (async_alloc(st) != 0 || reserve_events(st, st->gen + n_gens) != 0) return -2;
    const orc_config *c = &st->cfg;
    const uint32_t N = c->island_size, words = st->words;
    for (uint32_t isl = 0; isl < st->n_islands; ++isl) {
        for (uint32_t i = 0; i < n_gens; ++i) {
            const uint32_t g = (uint32_t)(st->gen + i);
            if (c->migrate_every != 0 && g % c->migrate_every == 0)
                async_migrate_island(st, isl, g, arrivals);
            reproduce_island(st, isl, g, NULL);
            /* the island's next population replaces its current one */
            const size_t base = (size_t)isl * N;
            memcpy(&st->trait[base], &st->trait2[base], N * sizeof(int32_t));
            memcpy(&st->counter[base], &st->counter2[base], N * sizeof(uint32_t));
            memcpy(&st->surface[base * words], &st->surface2[base * words],
                   (size_t)N * words * sizeof(uint32_t));
            if (tracking(st)) memcpy(&st->tag[base], &st->tag2[base], N * sizeof(int64_t));
        }
    }
    st->gen += n_gens;
    return 0;
}

/* Canonical agent record: int32 trait, uint32 counter, uint32 surface[words], zero padding
   up to a multiple of 16 bytes. */
uint32_t orc_record_bytes(const orc_state *st) { return ((8 + 4 * st->words) + 15) / 16 * 16; }

void orc_snapshot(const orc_state *st, void *dst)
{
    uint32_t rb = orc_record_bytes(st);
    uint8_t *out = (uint8_t *)dst;
    memset(out, 0, (size_t)rb * st->n_agents);
    for (uint32_t a = 0; a < st->n_agents; ++a) {
        uint8_t *rec = out + (size_t)a * rb;
        memcpy(rec, &st->trait[a], 4);
        memcpy(rec + 4, &st->counter[a], 4);
        memcpy(rec + 8, &st->surface[(size_t)a * st->words], 4 * st->words);
    }
}

void orc_load(orc_state *st, const void *src, uint64_t generation)
{
    uint32_t rb = orc_record_bytes(st);
    const uint8_t *in = (const uint8_t *)src;
    for (uint32_t a = 0; a < st->n_agents; ++a) {
        const uint8_t *rec = in + (size_t)a * rb;
        memcpy(&st->trait[a], rec, 4);
        memcpy(&st->counter[a], rec + 4, 4);
        memcpy(&st->surface[(size_t)a * st->words], rec + 8, 4 * st->words);
    }
    st->gen = generation;
    async_clear(st);
    if (tracking(st)) {
        for (uint32_t a = 0; a < st->n_agents; ++a) st->tag[a] = -1;
        for (uint32_t k = 0; k < st->n_islands * 4; ++k) st->mail_tag[k] = -1;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Lineage tracking (test support): the true divergence rank of two agents.              */
/* ------------------------------------------------------------------------------------ */

/* Start tracking: every current agent (and mailbox) becomes a root of the pedigree.
   Returns 0, or -2 when out of memory. */
int orc_track_lineage(orc_state *st)
{
    if (tracking(st)) return 0;
    st->tag = (int64_t *)malloc(st->n_agents * sizeof(int64_t));
    st->tag2 = (int64_t *)malloc(st->n_agents * sizeof(int64_t));
    st->mail_tag = (int64_t *)malloc((size_t)st->n_islands * 4 * sizeof(int64_t));
    if (!st->tag || !st->tag2 || !st->mail_tag) return -2;
    for (uint32_t a = 0; a < st->n_agents; ++a) st->tag[a] = st->tag2[a] = -1;
    for (uint32_t k = 0; k < st->n_islands * 4; ++k) st->mail_tag[k] = -1;
    return 0;
}

static uint32_t depth_of(const orc_state *st, int64_t e) { return e < 0 ? 0u : st->event_depth[e]; }

/*
 * D for each pair (i, j), i < j, row-major: the number of births the two agents' lineages
 * share (their latest common birth's child counter; 0 when they share none).  Deposits of
 * ranks below D were made once for both; the deposit of rank D, if both reach it, was drawn
 * in two separate births.  Returns 0, or -1 when tracking is off.
 */
int orc_divergence(const orc_state *st, const uint32_t *ids, uint32_t n, uint32_t *out)
{
    if (!tracking(st)) return -1;
    uint64_t p = 0;
    for (uint32_t i = 0; i < n; ++i)
        for (uint32_t j = i + 1; j < n; ++j, ++p) {
            int64_t a = st->tag[ids[i]], b = st->tag[ids[j]];
            while (a != b) {
                if (depth_of(st, a) >= depth_of(st, b)) a = st->event_parent[a];
                else b = st->event_parent[b];
            }
            out[p] = depth_of(st, a);
        }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Pairwise MRCA bounds (Fig. 1 caption: post hoc estimation of relatedness).            */
/* ------------------------------------------------------------------------------------ */

/* K = smallest integer with 2^(-b K) < 1 - confidence (confidence 0.95). */
uint32_t orc_mrca_margin(uint32_t b)
{
    uint32_t K = 1;
    while (pow(2.0, -(double)b * (double)K) >= 0.05) ++K;
    return K;
}

/* Site -> rank held at time T, by replaying the curation rule over ranks 0..T-1.  Sites
   that never received a deposit hold -1 (founder bits, shared by every agent). */
void orc_site_ranks(uint32_t policy, uint32_t S, uint64_t T, int64_t *rank_of_site)
{
    for (uint32_t k = 0; k < S; ++k) rank_of_site[k] = -1;
    for (uint64_t t = 0; t < T; ++t) {
        int64_t site = orc_site(policy, S, t);
        if (site >= 0) rank_of_site[site] = (int64_t)t;
    }
}

static uint32_t differentia(const uint8_t *rec, uint32_t site, uint32_t b)
{
    uint32_t pos = site * b, w;
    memcpy(&w, rec + 8 + 4 * (pos / 32), 4);
    return (w >> (pos % 32)) & ((1u << b) - 1u);
}

/*
 * For sampled agents (canonical records, all with counter T) and every pair i < j in
 * row-major upper-triangle order, bound the divergence rank D (the first rank whose
 * deposit the two lineages drew in separate births; ranks below D are shared by descent):
 *   retained ranks r_1 < ... < r_m (those < T held by some site); i* = first index whose
 *   differentiae differ.
 *   hi = r_{i*}                              (certain: a mismatch needs a separate draw)
 *   lo = r_{i*-K} + 1, or 0 when i* <= K     (K matches in a row by chance: prob 2^-bK)
 *   with no mismatch: hi = T, lo = r_{m-K+1} + 1 (0 when m < K).
 * Returns 0, or -1 when an agent's counter differs from T.
 */
int orc_mrca_bounds(const void *records, uint32_t record_bytes, const uint32_t *ids, uint32_t n,
                    uint32_t policy, uint32_t S, uint32_t b, uint64_t T, uint32_t *lo,
                    uint32_t *hi)
{
    const uint8_t *base = (const uint8_t *)records;
    int64_t *rank_of_site = (int64_t *)malloc(S * sizeof(int64_t));
    uint32_t *order = (uint32_t *)malloc(S * sizeof(uint32_t));
    if (!rank_of_site || !order) {
        free(rank_of_site);
        free(order);
        return -2;
    }
    orc_site_ranks(policy, S, T, rank_of_site);
    /* sites holding a rank, sorted by rank (selection sort: S is small) */
    uint32_t m = 0;
    for (uint32_t k = 0; k < S; ++k)
        if (rank_of_site[k] >= 0) order[m++] = k;
    for (uint32_t a = 0; a < m; ++a)
        for (uint32_t c = a + 1; c < m; ++c)
            if (rank_of_site[order[c]] < rank_of_site[order[a]]) {
                uint32_t t = order[a];
                order[a] = order[c];
                order[c] = t;
            }
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t cnt;
        memcpy(&cnt, base + (size_t)ids[i] * record_bytes + 4, 4);
        if ((uint64_t)cnt != T) {
            free(rank_of_site);
            free(order);
            return -1;
        }
    }
    const uint32_t K = orc_mrca_margin(b);
    uint64_t p = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const uint8_t *ra = base + (size_t)ids[i] * record_bytes;
        for (uint32_t j = i + 1; j < n; ++j, ++p) {
            const uint8_t *rb = base + (size_t)ids[j] * record_bytes;
            uint32_t first = 0; /* 1-based index of the first mismatch, 0 = none */
            for (uint32_t q = 0; q < m; ++q)
                if (differentia(ra, order[q], b) != differentia(rb, order[q], b)) {
                    first = q + 1;
                    break;
                }
            if (first) {
                hi[p] = (uint32_t)rank_of_site[order[first - 1]];
                lo[p] = first > K ? (uint32_t)rank_of_site[order[first - 1 - K]] + 1u : 0u;
            } else {
                hi[p] = (uint32_t)T;
                lo[p] = m >= K ? (uint32_t)rank_of_site[order[m - K]] + 1u : 0u;
            }
        }
    }
    free(rank_of_site);
    free(order);
    return 0;
}

/*
 * Pairwise MRCA bounds when the sampled agents' counters may differ (asynchronous runs: an
 * immigrant carries the counter of the island it was born in).  A rank r is only ever
 * deposited at site(r), so agents a and b (counters Ta, Tb) share rank r exactly when their
 * site -> rank tables at Ta and Tb hold r at the same site.  Over those common ranks, in rank
 * order c_1 < ... < c_m:
 *   first mismatch at c_{i*}: hi = c_{i*}, lo = c_{i*-K} + 1 (0 when i* <= K);
 *   no mismatch: hi = min(Ta, Tb), lo = c_{m-K+1} + 1 (0 when m < K).
 * With Ta = Tb this is orc_mrca_bounds.  Returns 0, or -2 when out of memory.
 */
typedef struct {
    uint64_t T;
    int64_t *table;
} rank_table;

static const int64_t *table_for(rank_table *cache, uint32_t *n_cached, uint32_t policy, uint32_t S,
                                uint64_t T)
{
    for (uint32_t i = 0; i < *n_cached; ++i)
        if (cache[i].T == T) return cache[i].table;
    int64_t *t = (int64_t *)malloc(S * sizeof(int64_t));
    if (!t) return NULL;
    orc_site_ranks(policy, S, T, t);
    cache[*n_cached].T = T;
    cache[*n_cached].table = t;
    *n_cached += 1;
    return t;
}

int orc_mrca_bounds_mixed(const void *records, uint32_t record_bytes, const uint32_t *ids,
                          uint32_t n, uint32_t policy, uint32_t S, uint32_t b, uint32_t *lo,
                          uint32_t *hi)
{
    const uint8_t *base = (const uint8_t *)records;
    rank_table *cache = (rank_table *)calloc(n ? n : 1, sizeof(rank_table));
    const int64_t **tab = (const int64_t **)calloc(n ? n : 1, sizeof(int64_t *));
    uint32_t *cnt = (uint32_t *)calloc(n ? n : 1, sizeof(uint32_t));
    int64_t *crank = (int64_t *)malloc(S * sizeof(int64_t));
    uint32_t *csite = (uint32_t *)malloc(S * sizeof(uint32_t));
    uint32_t n_cached = 0;
    int rc = 0;
    if (!cache || !tab || !cnt || !crank || !csite) rc = -2;
    for (uint32_t i = 0; i < n && rc == 0; ++i) {
        memcpy(&cnt[i], base + (size_t)ids[i] * record_bytes + 4, 4);
        tab[i] = table_for(cache, &n_cached, policy, S, cnt[i]);
        if (!tab[i]) rc = -2;
    }
    const uint32_t K = orc_mrca_margin(b);
    uint64_t p = 0;
    for (uint32_t i = 0; i < n && rc == 0; ++i) {
        const uint8_t *ra = base + (size_t)ids[i] * record_bytes;
        for (uint32_t j = i + 1; j < n; ++j, ++p) {
            const uint8_t *rb = base + (size_t)ids[j] * record_bytes;
            /* common ranks, sorted ascending (insertion sort: S is small) */
            uint32_t m = 0;
            for (uint32_t k = 0; k < S; ++k) {
                if (tab[i][k] < 0 || tab[i][k] != tab[j][k]) continue;
                uint32_t q = m++;
                while (q > 0 && crank[q - 1] > tab[i][k]) {
                    crank[q] = crank[q - 1];
                    csite[q] = csite[q - 1];
                    --q;
                }
                crank[q] = tab[i][k];
                csite[q] = k;
            }
            uint32_t first = 0;
            for (uint32_t q = 0; q < m; ++q)
                if (differentia(ra, csite[q], b) != differentia(rb, csite[q], b)) {
                    first = q + 1;
                    break;
                }
            if (first) {
                hi[p] = (uint32_t)crank[first - 1];
                lo[p] = first > K ? (uint32_t)crank[first - 1 - K] + 1u : 0u;
            } else {
                hi[p] = cnt[i] < cnt[j] ? cnt[i] : cnt[j];
                lo[p] = m >= K ? (uint32_t)crank[m - K] + 1u : 0u;
            }
        }
    }
    for (uint32_t i = 0; i < n_cached; ++i) free(cache[i].table);
    free(cache);
    free(tab);
    free(cnt);
    free(crank);
    free(csite);
    return rc;
}

/* Oracle-side state accessors for tests. */
const int32_t *orc_traits(const orc_state *st) { return st->trait; }
const uint32_t *orc_counters(const orc_state *st) { return st->counter; }
uint32_t orc_surface_words(const orc_state *st) { return st->words; }
int orc_openmp_enabled(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}
