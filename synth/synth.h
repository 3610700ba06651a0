/* Seeded synthetic metagenome read generator (input recipe only). */
#ifndef SYNTH_H
#define SYNTH_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    uint64_t seed;
    uint32_t n_genomes;
    uint64_t genome_len_min, genome_len_max;  /* uniform genome length */
    double abundance_sigma;                   /* log-normal sigma; 0 = equal */
    uint64_t n_reads;
    uint32_t read_len_min, read_len_max;      /* uniform read length */
    double subst_rate;                        /* substitution probability per base */
    int err_qual_lo, err_qual_hi;             /* Phred of substituted bases; lo < 0 = same law as the rest */
    double qual_mean, qual_sd;                /* Phred ~ round(N(mean, sd)) clipped */
    int qual_min, qual_max;
    double n_rate;                            /* probability that a base reads as N */
    int n_qual;                               /* Phred given to N bases */
    int qual_offset;                          /* 33 = FASTQ ASCII */
    int n_threads;
} synth_params;

int synth_genome_lengths(const synth_params *p, uint64_t *lens);
int synth_genomes(const synth_params *p, const uint64_t *lens, char *seq);
int synth_read_offsets(const synth_params *p, uint64_t *offsets);
int synth_reads(const synth_params *p, const uint64_t *lens, const char *genomes,
                const uint64_t *offsets, char *bases, uint8_t *quals,
                uint32_t *truth_genome, uint64_t *truth_pos, uint8_t *truth_strand);

#ifdef __cplusplus
}
#endif
#endif
