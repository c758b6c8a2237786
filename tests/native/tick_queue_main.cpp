// Prints the persistent tick's work queue for the stream sizes given on the
// command line, for the CPU tests of its order (tests/test_tick_queue_cpu.py).
// usage: tick_queue_main piece lag w0 h0 w1 h1 ...
// output: "rows R" (the strip height), one line per item "kind stream begin
// end", then one line per stream "sync nl nc nm".
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "hmi_queue.h"

int main(int argc, char **argv)
{
    if (argc < 5 || (argc - 3) % 2 != 0) return 2;
    const int piece = std::atoi(argv[1]);
    const long long lag = std::atoll(argv[2]);
    std::vector<int> chunks, strips;
    for (int i = 3; i + 1 < argc; i += 2) {
        const int w = std::atoi(argv[i]), h = std::atoi(argv[i + 1]);
        const int nwords = (w + 31) / 32, strips_x = (nwords + 29) / 30;
        chunks.push_back(h * 2 * nwords);
        strips.push_back(((h + hmi::kStripRows - 1) / hmi::kStripRows) * strips_x);
    }
    std::vector<hmi::TickSync> sync;
    const std::vector<int4> q = hmi::tick_queue(chunks, strips, piece, lag, &sync);
    std::printf("rows %d\n", hmi::kStripRows);
    for (const int4 &e : q) std::printf("%d %d %d %d\n", e.x >> 24, e.x & 0xffffff, e.y, e.z);
    for (const hmi::TickSync &y : sync) std::printf("sync %u %u %u\n", y.nl, y.nc, y.nm);
    return 0;
}
