/*
 * int_rates.h -- integer pipe-rate probes of liblinac_probes.so, the
 * benchmark's measurement library (not part of liblinac.so; the paper has no
 * counterpart).  They give the measured roofline denominators of the
 * trailing-update paths on the current device.
 */
#ifndef LINAC_PROBES_INT_RATES_H
#define LINAC_PROBES_INT_RATES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *cudaStream_t;

typedef struct {
    double imad_wide_per_s;     /* thread-level mad.wide.s32 per second (plain path) */
    double imma_u8_mac_per_s;   /* u8 multiply-adds per second of mma.sync m16n8k32 (limb path) */
    double dp4a_u8_mac_per_s;   /* u8 multiply-adds per second of dp4a */
    double sm_clock_khz;        /* nominal maximum SM clock */
    int sm_count;
    /* one block of 512 threads per SM: warps 0-7 run mad.wide.s32, warps 8-15
     * mma.sync u8; time with only the first group working, only the second,
     * and both at once (ms) */
    double coissue_imad_only_ms;
    double coissue_imma_only_ms;
    double coissue_both_ms;
    double imma_s8_mac_per_s;   /* s8 multiply-adds per second of mma.sync m16n8k32 (multi-modular path) */
} linac_int_rates;

/* Runs the probes on the current device (allocates a small buffer and
 * synchronises `stream`).  Returns 0 on success, 1 for a null pointer, 4 for a
 * CUDA error, 5 if the buffer could not be allocated. */
int linac_probe_int_rates(linac_int_rates *out, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif
