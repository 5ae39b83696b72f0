// Host build of the float-float header (plain C++, no CUDA), driven by
// tests/test_ff_host.py.  Reads one operation per line from stdin,
//
//   two_sum a b | fast_two_sum a b | add ah al bh bl | sub ah al bh bl |
//   mul ah al bh bl | rcp ah al | from_d d
//
// with every operand a C99 hexadecimal float, and prints the result's hi and
// lo words in the same notation (%a), one line per operation.  Must be built
// with -ffp-contract=off.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "ff.cuh"

using mba::ff;

namespace {

bool read_f(float *v) {
    char buf[64];
    if (std::scanf("%63s", buf) != 1) return false;
    *v = std::strtof(buf, nullptr);
    return true;
}

bool read_ff(ff *v) { return read_f(&v->hi) && read_f(&v->lo); }

}  // namespace

int main() {
    char op[32];
    while (std::scanf("%31s", op) == 1) {
        ff r{0.f, 0.f}, a{0.f, 0.f}, b{0.f, 0.f};
        bool ok = true;
        if (!std::strcmp(op, "two_sum") || !std::strcmp(op, "fast_two_sum")) {
            ok = read_f(&a.hi) && read_f(&b.hi);
            r = op[0] == 't' ? mba::ff_two_sum(a.hi, b.hi) : mba::ff_fast_two_sum(a.hi, b.hi);
        } else if (!std::strcmp(op, "add") || !std::strcmp(op, "sub") || !std::strcmp(op, "mul")) {
            ok = read_ff(&a) && read_ff(&b);
            r = op[0] == 'a' ? mba::ff_add(a, b) : op[0] == 's' ? mba::ff_sub(a, b) : mba::ff_mul(a, b);
        } else if (!std::strcmp(op, "rcp")) {
            ok = read_ff(&a);
            r = mba::ff_rcp(a);
        } else if (!std::strcmp(op, "from_d")) {
            char buf[64];
            ok = std::scanf("%63s", buf) == 1;
            r = mba::ff_from(std::strtod(buf, nullptr));
        } else {
            ok = false;
        }
        if (!ok) {
            std::fprintf(stderr, "bad input at operation '%s'\n", op);
            return 2;
        }
        std::printf("%a %a\n", (double)r.hi, (double)r.lo);
    }
    return 0;
}
