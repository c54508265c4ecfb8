/*
 * pcpd_decay.c -- a plain C user of libpcpd.so (include/pcpd.h): a decay run of the PCPD
 * (or, with a fifth argument 3 or 4, of the TCPD / QCPD) from a fully occupied ring, printing
 * the particle and pair densities at log-spaced MCS times.
 *
 *   pcpd_decay L samples p d [tuple] [mcs] [seed]
 *
 * Output: one line per record, "t rho rho_pair".  Exit status 0 on success, else the
 * library's error code with its message on stderr.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "pcpd.h"

static int check(int rc)
{
    if (rc != PCPD_OK) fprintf(stderr, "pcpd error %d: %s\n", rc, pcpd_last_error());
    return rc;
}

int main(int argc, char **argv)
{
    if (argc < 5) {
        fprintf(stderr, "usage: %s L samples p d [tuple] [mcs] [seed]\n", argv[0]);
        return 1;
    }
    pcpd_params prm;
    memset(&prm, 0, sizeof prm);
    prm.L = (uint32_t)strtoul(argv[1], NULL, 10);
    prm.samples = (uint32_t)strtoul(argv[2], NULL, 10);
    prm.p = atof(argv[3]);
    prm.d = atof(argv[4]);
    prm.tuple = argc > 5 ? (uint32_t)strtoul(argv[5], NULL, 10) : 0u;
    const uint64_t mcs = argc > 6 ? strtoull(argv[6], NULL, 10) : 1000u;
    prm.seed = argc > 7 ? strtoull(argv[7], NULL, 10) : 1u;
    prm.init = PCPD_INIT_FULL;

    /* strictly increasing log-spaced times 1 .. mcs */
    enum { R = 24 };
    uint64_t t[R];
    size_t n = 0;
    for (int k = 0; k < R; ++k) {
        uint64_t v = (uint64_t)ceil(pow((double)mcs, (double)k / (R - 1)));
        if (n && v <= t[n - 1]) v = t[n - 1] + 1;
        if (v > mcs) break;
        t[n++] = v;
    }

    pcpd_t *h = NULL;
    int rc = check(pcpd_create_ex(&prm, &h));
    if (rc) return rc;
    rc = check(pcpd_run(h, mcs, t, n));
    double rho[R];
    uint64_t pairs[R];
    if (!rc) rc = check(pcpd_density(h, rho, NULL, n));
    if (!rc) rc = check(pcpd_pair_counts(h, pairs, n));
    if (!rc)
        for (size_t r = 0; r < n; ++r)
            printf("%llu %.9f %.9f\n", (unsigned long long)t[r], rho[r],
                   (double)pairs[r] / ((double)prm.L * prm.samples));
    pcpd_destroy(h);
    return rc;
}
