/*
 * Seeded synthetic metagenome reads: the input recipe shared by the oracle,
 * the CUDA path, the tests and the benchmark.  This file holds none of the
 * k-mer analysis arithmetic: it only draws genomes, read placements,
 * sequencing errors and Phred qualities.
 *
 * The recipe follows the MGSim description of the paper (Sec. IV-A,
 * "Experimental Datasets"): several random genomes, each with a relative
 * abundance drawn from a log-normal law, reads sampled from both strands with
 * uniform substitution errors (wgsim style).  Every random number is drawn
 * from a per-item counter-based stream (splitmix64 seeding xoshiro256**, both
 * published generators), so any read can be regenerated alone and the output
 * does not depend on the number of threads.
 *
 * Build with -ffp-contract=off so that x86 and Arm give identical bytes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "synth.h"

/* splitmix64 (Steele, Lea, Flood 2014). */
static uint64_t sm64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* xoshiro256** (Blackman, Vigna 2018). */
typedef struct { uint64_t s[4]; } rng_t;
static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t res = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return res;
}
/* Independent stream for (seed, domain, index). */
static void rng_seed(rng_t *r, uint64_t seed, uint64_t domain, uint64_t index) {
    uint64_t x = seed ^ (domain * 0xD1B54A32D192ED03ull) ^ (index * 0x8CB92BA72F3D8DD7ull);
    sm64(&x);
    for (int i = 0; i < 4; ++i) r->s[i] = sm64(&x);
}
static double rng_unif(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }
static uint64_t rng_below(rng_t *r, uint64_t n) { /* n >= 1; multiply-shift, bias < 2^-64 * n */
    return (uint64_t)(((unsigned __int128)rng_next(r) * n) >> 64);
}
/* Approximate standard normal: Irwin-Hall sum of 12 uniforms minus 6 (pure
 * additions, so bit-identical on every IEEE machine). */
static double rng_normal(rng_t *r) {
    double s = 0.0;
    for (int i = 0; i < 12; ++i) s += rng_unif(r);
    return s - 6.0;
}

enum { DOM_GLEN = 1, DOM_GSEQ = 2, DOM_ABUND = 3, DOM_READ = 4, DOM_RLEN = 5 };

static const char BASES[4] = {'A', 'C', 'G', 'T'};

static int check_params(const synth_params *p) {
    if (!p) return -1;
    if (p->n_genomes == 0 || p->genome_len_min == 0 || p->genome_len_max < p->genome_len_min) return -1;
    if (p->read_len_min == 0 || p->read_len_max < p->read_len_min) return -1;
    if (p->read_len_max > p->genome_len_min) return -1;  /* every read must fit in every genome */
    if (p->qual_min < 0 || p->qual_max < p->qual_min || p->qual_max > 93) return -1;
    return 0;
}

int synth_genome_lengths(const synth_params *p, uint64_t *lens) {
    if (check_params(p) || !lens) return -1;
    for (uint32_t g = 0; g < p->n_genomes; ++g) {
        rng_t r; rng_seed(&r, p->seed, DOM_GLEN, g);
        uint64_t span = p->genome_len_max - p->genome_len_min + 1;
        lens[g] = p->genome_len_min + rng_below(&r, span);
    }
    return 0;
}

static uint32_t read_length(const synth_params *p, uint64_t i) {
    if (p->read_len_min == p->read_len_max) return p->read_len_min;
    rng_t r; rng_seed(&r, p->seed, DOM_RLEN, i);
    return p->read_len_min + (uint32_t)rng_below(&r, (uint64_t)(p->read_len_max - p->read_len_min) + 1);
}

int synth_read_offsets(const synth_params *p, uint64_t *offsets) {
    if (check_params(p) || !offsets) return -1;
    offsets[0] = 0;
    for (uint64_t i = 0; i < p->n_reads; ++i) offsets[i + 1] = offsets[i] + read_length(p, i);
    return 0;
}

int synth_genomes(const synth_params *p, const uint64_t *lens, char *seq) {
    if (check_params(p) || !lens || !seq) return -1;
    uint64_t off = 0;
    for (uint32_t g = 0; g < p->n_genomes; ++g) {
        rng_t r; rng_seed(&r, p->seed, DOM_GSEQ, g);
        uint64_t L = lens[g];
        uint64_t i = 0;
        while (i < L) { /* 32 bases per draw */
            uint64_t x = rng_next(&r);
            for (int j = 0; j < 32 && i < L; ++j, ++i) { seq[off + i] = BASES[x & 3]; x >>= 2; }
        }
        off += L;
    }
    return 0;
}

static unsigned char comp_char(char c) {
    switch (c) { case 'A': return 'T'; case 'C': return 'G'; case 'G': return 'C'; case 'T': return 'A'; }
    return 'N';
}

static int draw_qual(const synth_params *p, rng_t *r) {
    double q = nearbyint(p->qual_mean + p->qual_sd * rng_normal(r));
    if (q < p->qual_min) q = p->qual_min;
    if (q > p->qual_max) q = p->qual_max;
    return (int)q;
}

int synth_reads(const synth_params *p, const uint64_t *lens, const char *genomes,
                const uint64_t *offsets, char *bases, uint8_t *quals,
                uint32_t *truth_genome, uint64_t *truth_pos, uint8_t *truth_strand) {
    if (check_params(p) || !lens || !genomes || !offsets || !bases || !quals) return -1;
    uint32_t G = p->n_genomes;
    double *cum = (double *)malloc(sizeof(double) * G);
    uint64_t *gstart = (uint64_t *)malloc(sizeof(uint64_t) * G);
    if (!cum || !gstart) { free(cum); free(gstart); return -2; }
    /* read source chosen in proportion to abundance x length, so that each
     * genome's coverage is proportional to its abundance */
    double tot = 0.0;
    uint64_t s = 0;
    for (uint32_t g = 0; g < G; ++g) {
        double a = 1.0;
        if (p->abundance_sigma > 0.0) {
            rng_t r; rng_seed(&r, p->seed, DOM_ABUND, g);
            a = exp(p->abundance_sigma * rng_normal(&r));
        }
        tot += a * (double)lens[g];
        cum[g] = tot;
        gstart[g] = s;
        s += lens[g];
    }
    int64_t n = (int64_t)p->n_reads;
#pragma omp parallel for schedule(static, 4096) num_threads(p->n_threads > 0 ? p->n_threads : 1)
    for (int64_t i = 0; i < n; ++i) {
        rng_t r; rng_seed(&r, p->seed, DOM_READ, (uint64_t)i);
        uint64_t L = offsets[i + 1] - offsets[i];
        double u = rng_unif(&r) * tot;
        uint32_t lo = 0, hi = G - 1;
        while (lo < hi) { uint32_t mid = (lo + hi) / 2; if (cum[mid] > u) hi = mid; else lo = mid + 1; }
        uint32_t g = lo;
        uint64_t pos = rng_below(&r, lens[g] - L + 1);
        int strand = (int)(rng_next(&r) & 1);
        const char *src = genomes + gstart[g] + pos;
        char *dst = bases + offsets[i];
        uint8_t *qd = quals + offsets[i];
        for (uint64_t j = 0; j < L; ++j) {
            char c = strand ? (char)comp_char(src[L - 1 - j]) : src[j];
            int q = draw_qual(p, &r);
            double e = rng_unif(&r);
            if (e < p->subst_rate) {
                int cur = c == 'A' ? 0 : c == 'C' ? 1 : c == 'G' ? 2 : 3;
                int alt = (cur + 1 + (int)rng_below(&r, 3)) & 3;
                c = BASES[alt];
                if (p->err_qual_lo >= 0)
                    q = p->err_qual_lo + (int)rng_below(&r, (uint64_t)(p->err_qual_hi - p->err_qual_lo + 1));
            } else if (e < p->subst_rate + p->n_rate) {
                c = 'N';
                q = p->n_qual;
            }
            dst[j] = c;
            qd[j] = (uint8_t)(q + p->qual_offset);
        }
        if (truth_genome) truth_genome[i] = g;
        if (truth_pos) truth_pos[i] = pos;
        if (truth_strand) truth_strand[i] = (uint8_t)strand;
    }
    free(cum);
    free(gstart);
    return 0;
}
