/*
 * rng_stdout: the paper's example program (Section 5) written against the C
 * ABI in include/rng.h.  Usage: rng_stdout n i [seed] > out.bin
 * Writes i iterations of n 64-bit values as raw binary to stdout (8*n*i
 * bytes, Eq. 1) and the profiling summary to stderr.
 */
#include <stdio.h>
#include <stdlib.h>
#include <unistd.h>

#include "rng.h"

static int report(rng_err **err) {
    fprintf(stderr, "rng_stdout: %s\n", *err ? (*err)->msg : "error");
    rng_err_clear(err);
    return EXIT_FAILURE;
}

int main(int argc, char **argv) {
    if (argc < 3) {
        fprintf(stderr, "usage: %s n i [seed]\n", argv[0]);
        return EXIT_FAILURE;
    }
    const unsigned long long n = strtoull(argv[1], NULL, 10);
    const unsigned long long iters = strtoull(argv[2], NULL, 10);
    const unsigned long long seed = argc > 3 ? strtoull(argv[3], NULL, 10) : 0;

    rng_err *err = NULL;
    rng_opts opts;
    rng_opts_default(&opts);
    opts.host_path = 1; /* device-side double buffer, as in the paper */

    rng_gen *g = NULL;
    if (rng_create(n, seed, &opts, &g, &err) != RNG_OK) return report(&err);
    if (rng_init(g, &err) != RNG_OK || rng_generate_fd(g, iters, STDOUT_FILENO, &err) != RNG_OK) {
        rng_destroy(g);
        return report(&err);
    }
    const char *summary = rng_profile_summary(g, RNG_PROF_SORT_TIME | RNG_PROF_SORT_DESC,
                                              RNG_PROF_SORT_TIME | RNG_PROF_SORT_DESC, &err);
    if (summary) fputs(summary, stderr);
    rng_destroy(g);
    if (rng_live_objects() != 0) fprintf(stderr, "rng_stdout: objects left alive\n");
    return summary ? EXIT_SUCCESS : report(&err);
}
