"""Host-side check of the device error word's status mapping (no GPU): every
condition has a bit of its own, and each bit maps to the status and message the
C ABI documents.  The mapping header is plain C++; it is compiled here with g++
into a small harness that prints the status of each error word."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2002_00054_b300", "csrc", "error_word.h")

HARNESS = r'''
#include "%s"
#include <cstdio>
int main() {
    const int bits[] = {ERR_NEIGH_OVERFLOW, ERR_CELL_OVERFLOW, ERR_NONFINITE, ERR_CLOSE, ERR_REV,
                        ERR_RC_OVERFLOW, ERR_RANGE, ERR_TIMEOUT};
    const char* names[] = {"NEIGH_OVERFLOW", "CELL_OVERFLOW", "NONFINITE", "CLOSE", "REV",
                           "RC_OVERFLOW", "RANGE", "TIMEOUT"};
    int all = 0;
    for (int k = 0; k < 8; ++k) {
        char msg[256];
        const int st = error_word_status(bits[k], 192, 256, 32000.0, msg, sizeof msg);
        printf("%%s %%d %%d %%s\n", names[k], bits[k], st, msg);
        all |= bits[k];
    }
    printf("ALL %%d %%d\n", all, ERR_ALL_BITS);
    for (int f = 1; f <= ERR_ALL_BITS; ++f) {
        char msg[256];
        printf("W %%d %%d\n", f, error_word_status(f, 192, 256, 32000.0, msg, sizeof msg));
    }
    return 0;
}
'''


@pytest.fixture(scope="module")
def table(tmp_path_factory):
    d = tmp_path_factory.mktemp("errword")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS % HDR)
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)]).decode().splitlines()
    single, words = {}, {}
    for line in out:
        p = line.split(" ", 3)
        if p[0] == "W":
            words[int(p[1])] = int(p[2])
        elif p[0] == "ALL":
            single["ALL"] = (int(p[1]), int(p[2]))
        else:
            single[p[0]] = (int(p[1]), int(p[2]), p[3])
    return single, words


def test_bits_are_distinct_powers_of_two(table):
    single, _ = table
    bits = [v[0] for k, v in single.items() if k != "ALL"]
    assert len(set(bits)) == len(bits)
    assert all(b > 0 and (b & (b - 1)) == 0 for b in bits)
    assert single["ALL"][0] == single["ALL"][1]


def test_each_bit_maps_to_its_status(table):
    from paper_2002_00054_b300 import _capi as c
    single, _ = table
    want = {"NEIGH_OVERFLOW": c.NNP_ENEIGH_OVERFLOW, "CELL_OVERFLOW": c.NNP_ENEIGH_OVERFLOW,
            "NONFINITE": c.NNP_ENONFINITE, "CLOSE": c.NNP_ENONFINITE, "REV": c.NNP_ECUDA,
            "RC_OVERFLOW": c.NNP_ECUDA, "RANGE": c.NNP_ENONFINITE, "TIMEOUT": c.NNP_ECUDA}
    for name, status in want.items():
        assert single[name][1] == status, name
    # the tensor-core timeout is not reported as a physics (force-range) error
    assert "tensor-core" in single["TIMEOUT"][2] and "force" not in single["TIMEOUT"][2]
    assert "max_neighbors = 192" in single["NEIGH_OVERFLOW"][2]


def test_timeout_outranks_numerical_conditions(table):
    from paper_2002_00054_b300 import _capi as c
    single, words = table
    t = single["TIMEOUT"][0]
    for name in ("RANGE", "CLOSE", "NONFINITE"):
        assert words[t | single[name][0]] == c.NNP_ECUDA
    assert words[t | single["NEIGH_OVERFLOW"][0]] == c.NNP_ENEIGH_OVERFLOW
    assert all(v != c.NNP_OK for v in words.values())
