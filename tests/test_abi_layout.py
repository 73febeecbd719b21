"""The Python binding's ctypes structures have the C ABI's layout: for every
struct of include/pic.h and include/pic_owmr.h, gcc compiles the headers and
prints sizeof and each member's offset, which must equal the ctypes field
offsets and sizes (no GPU needed)."""
import os
import subprocess
import tempfile

import pytest

import paper_2406_01939_b300 as pic
from paper_2406_01939_b300 import owmr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = [pic.pic_instance_desc, pic.pic_policy, pic.pic_sim_opts, pic.pic_sim_result,
           pic.pic_traj_result, pic.pic_grad_args, owmr.pic_owmr_desc, owmr.pic_owmr_policy,
           owmr.pic_owmr_opts, owmr.pic_owmr_result]


def c_layout():
    """{struct: (sizeof, {member: offset})} as gcc lays the headers out."""
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pic.h"',
             '#include "pic_owmr.h"', "int main(void) {"]
    for S in STRUCTS:
        n = S.__name__
        lines.append(f'printf("{n} sizeof %zu\\n", sizeof({n}));')
        for f in S._fields_:
            lines.append(f'printf("{n} {f[0]} %zu\\n", offsetof({n}, {f[0]}));')
    lines += ["return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                       check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    lay = {}
    for line in out.splitlines():
        n, m, v = line.split()
        size, offs = lay.setdefault(n, [0, {}])
        if m == "sizeof":
            lay[n][0] = int(v)
        else:
            offs[m] = int(v)
    return lay


@pytest.mark.parametrize("S", STRUCTS, ids=lambda S: S.__name__)
def test_ctypes_struct_matches_c_layout(S):
    size, offs = c_layout()[S.__name__]
    assert {f[0] for f in S._fields_} == set(offs), "member names differ"
    for name, _ in S._fields_:
        assert getattr(S, name).offset == offs[name], name
    assert __import__("ctypes").sizeof(S) == size


def test_mode_constants_match_the_header():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    for name in ("PIC_MODE_PICARD", "PIC_MODE_SEQUENTIAL", "PIC_MODE_PICARD_PRODUCTS",
                 "PIC_MODE_PICARD_ASSIGNED"):
        v = int(src.split(name + " = ")[1].split(",")[0].split()[0])
        assert getattr(pic, name) == v, name
