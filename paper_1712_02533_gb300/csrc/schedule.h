// Host-side scan schedules of libreg.
#pragma once
#include <vector>

namespace regsched {

enum { OP_COMBINE = 0, OP_COPY = 1, OP_IDENTITY = 2 };
enum { K_SERIAL = 0, K_SKLANSKY = 1, K_KOGGE_STONE = 2, K_BRENT_KUNG = 3, K_BLELLOCH = 4, K_CHUNKED = 5,
       K_CHUNKED_ALT = 6, K_HAN_CARLSON = 7, K_LADNER_FISCHER = 8 };

struct Op {
    int kind, dst, a, b;
};

struct Schedule {
    std::vector<std::vector<Op>> levels;
};

// chunks: the chunk count of the chunked kinds, the parameter k of Han-Carlson
// and Ladner-Fischer
bool make_schedule(int kind, int n, int chunks, int global_kind, Schedule &out);
int aux_slots(int kind, int n, int chunks, int global_kind);

}  // namespace regsched
