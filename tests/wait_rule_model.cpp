// Host model of the kernels' bounded-wait loop (mbar_wait in the library's
// device header), driven by the same decision rule (fe_wait.h): a barrier
// phase completes at a given time; one probe suspends the thread until the
// phase completes or the suspend hint passes.  Prints, for the scenario named
// on the command line, "gave_up <n>" (waits that gave up) and "elapsed <ns>".
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../paper_2410_12614_gb300/csrc/fe_wait.h"

static unsigned long long now_ns = 0;

// one try_wait probe of a phase completing at `done`
static bool probe(unsigned long long done, uint32_t hint) {
    if (done <= now_ns) return true;
    if (done <= now_ns + hint) {
        now_ns = done;
        return true;
    }
    now_ns += hint;
    return false;
}

// the device loop: fast probe, then the clock and the limit
static bool bounded_wait(unsigned long long done, unsigned long long limit) {
    const uint32_t hint = fe::wait_suspend_hint(limit);
    if (probe(done, hint)) return true;
    const unsigned long long t0 = now_ns;
    while (!probe(done, hint)) {
        if (fe::wait_expired(t0, now_ns, limit)) return false;
    }
    return true;
}

int main(int argc, char **argv) {
    const char *sc = argc > 1 ? argv[1] : "long";
    const unsigned long long limit = argc > 2 ? strtoull(argv[2], nullptr, 10) : 2000000000ull;
    long gave_up = 0;
    if (!strcmp(sc, "long")) {
        // a persistent CTA: 100,000 waits, each satisfied 0.9 limit after it
        // starts, 50 us of work between them -- 45,000 limits in total
        for (int i = 0; i < 100000; ++i) {
            now_ns += 50000;
            if (!bounded_wait(now_ns + limit / 10 * 9, limit)) ++gave_up;
        }
    } else if (!strcmp(sc, "stall")) {
        // one wait whose phase never completes
        if (!bounded_wait(~0ull, limit)) ++gave_up;
    } else if (!strcmp(sc, "late")) {
        // a phase completing 3 limits + 3 hints after the wait began: too late
        const unsigned long long h = fe::wait_suspend_hint(limit);
        if (!bounded_wait(now_ns + 3 * limit + 3 * h, limit)) ++gave_up;
    }
    printf("gave_up %ld\nelapsed %llu\n", gave_up, now_ns);
    return 0;
}
