/*
 * dpm_host.h -- host-only inspection of the tables the library builds
 * (no GPU needed).  Used by the CPU tests to check the table builder against
 * the model's closed forms; not needed for transport.
 *
 * The tables are the FP32 data the transport kernels interpolate (Sec. 2.3 of
 * the paper keeps cross sections as tables in texture memory; here they are
 * plain arrays).
 */
#ifndef DPM_HOST_H
#define DPM_HOST_H

#include "dpm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Build the tables on the host.  Returns a handle, or NULL with a message in
   err (at least 256 bytes) when the arguments are invalid. */
void *dpm_host_tables_build(const dpm_material *mats, int n_mat, const dpm_table_params *p, char *err);
void dpm_host_tables_free(void *handle);

/* Copy table `name` ("ph", "el", "pmol", "kn", "mol", "brem", "pair", "msc")
   into out (at most n floats; out may be NULL to query the length).  meta
   (6 doubles, may be NULL) receives [e_lo, e_hi, rows or nodes, row or
   argument range lo, hi, columns].  Returns the table length or -1. */
int dpm_host_tables_get(void *handle, const char *name, float *out, int n, double *meta);

#ifdef __cplusplus
}
#endif
#endif
