"""User-defined tunable kernels (the kernel definition of Sec. 4.1 for any
kernel), host side: configuration space and restrictions, configuration
text, the integer-expression language of restrictions and launch geometry
(checked against Python's own integer arithmetic), and NVRTC compiles of
extern "C" and templated functions, without a GPU."""

from __future__ import annotations

import pytest

from paper_2303_12374_gb300 import kl

VADD = r"""
extern "C" __global__ void vadd(const float *a, const float *b, float *c, int n)
{
    // ELEMS strided chunks of BLOCK consecutive elements per block
    long base = (long)blockIdx.x * BLOCK * ELEMS + threadIdx.x;
#pragma unroll
    for (int e = 0; e < ELEMS; ++e) {
        long i = base + (long)e * BLOCK;
        if (i < n) c[i] = a[i] + b[i];
    }
}
"""

SCALE = r"""
template <int F>
__global__ void scale(float *x, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] *= F;
}
"""


def vadd_def():
    d = kl.KernelDef("vadd", VADD, "vadd")
    d.param("BLOCK", [32, 64, 128, 256, 512, 1024], 256)
    d.param("ELEMS", [1, 2, 4, 8], 1)
    d.restrict("BLOCK * ELEMS <= 4096")
    d.geometry(block=("BLOCK",), grid=("div_ceil(problem_x, BLOCK * ELEMS)",))
    return d


def test_space_and_restrictions():
    d = vadd_def()
    assert d.space_size() == (24, 23)            # only BLOCK=1024, ELEMS=8 breaks the restriction
    assert d.config_at(0) == ("BLOCK=32,ELEMS=1", True)
    assert d.config_at(5) == ("BLOCK=1024,ELEMS=1", True)
    assert d.config_at(6) == ("BLOCK=32,ELEMS=2", True)
    assert d.config_at(23) == ("BLOCK=1024,ELEMS=8", False)
    with pytest.raises(kl.KLError):
        d.config_at(24)


def test_configuration_text():
    d = vadd_def()
    assert d.normalize("default") == "BLOCK=256,ELEMS=1"
    assert d.normalize("ELEMS=4") == "BLOCK=256,ELEMS=4"
    assert d.normalize("ELEMS=2,BLOCK=64") == "BLOCK=64,ELEMS=2"
    for bad in ["FOO=1", "BLOCK=100", "BLOCK=64,BLOCK=64", "BLOCK", "BLOCK=x",
                "BLOCK=1024,ELEMS=8"]:
        with pytest.raises(kl.KLError) as e:
            d.normalize(bad)
        assert e.value.status == -1, bad


def test_geometry():
    d = vadd_def()
    assert d.launch_geometry("BLOCK=128,ELEMS=2", (1000,)) == [128, 1, 1, 4, 1, 1, 0]
    assert d.launch_geometry("default", (1,)) == [256, 1, 1, 1, 1, 1, 0]
    # defaults: block 1, grid = problem
    e = kl.KernelDef("e", "extern \"C\" __global__ void k() {}", "k")
    assert e.launch_geometry("default", (5, 6, 7)) == [1, 1, 1, 5, 6, 7, 0]
    # a problem of size 0 has no grid; more than 1024 threads do not apply
    with pytest.raises(kl.KLError):
        d.launch_geometry("default", (0,))
    big = kl.KernelDef("big", VADD, "vadd").param("B", [2048]).geometry(block=("B",))
    with pytest.raises(kl.KLError):
        big.launch_geometry("default", (10,))


EXPRS = [
    ("A * B + problem_x % 7", lambda A, B, x: A * B + x % 7),
    ("A < B ? A : B", lambda A, B, x: A if A < B else B),
    ("min(A, B) * max(A, B) - 1", lambda A, B, x: min(A, B) * max(A, B) - 1),
    ("div_ceil(problem_x, A)", lambda A, B, x: -(-x // A)),
    ("round_up(problem_x, B)", lambda A, B, x: -(-x // B) * B),
    ("(A | B) ^ (A & B)", lambda A, B, x: (A | B) ^ (A & B)),
    ("!(A == B) + (A != B) + (A <= B) + (A >= B) + (A > B)",
     lambda A, B, x: (A != B) * 2 + (A <= B) + (A >= B) + (A > B)),
    ("-A + ~B + 100", lambda A, B, x: -A + ~B + 100),
    ("A && B || 0", lambda A, B, x: 1),
    ("problem_x / A / B", lambda A, B, x: x // A // B),
    ("2 + 3 * 4 - 10 / 2 % 3", lambda A, B, x: 2 + 3 * 4 - 10 // 2 % 3),
    ("A > 3 ? B > 5 ? 1 : 2 : 3", lambda A, B, x: (1 if B > 5 else 2) if A > 3 else 3),
]


@pytest.mark.parametrize("expr,ref", EXPRS)
def test_expression_language(expr, ref):
    for A in (3, 5):
        for B in (2, 7):
            d = kl.KernelDef("x", "extern \"C\" __global__ void k() {}", "k")
            d.param("A", [A]).param("B", [B]).geometry(shared_memory=expr)
            for x in (1, 100, 1001):
                assert d.launch_geometry("default", (x,))[6] == ref(A, B, x), (expr, A, B, x)


@pytest.mark.parametrize("bad", ["A +", "A * (B", "FOO > 1", "min(A)", "pow(A, B)", "A $ B", ""])
def test_restriction_errors(bad):
    d = kl.KernelDef("x", "extern \"C\" __global__ void k() {}", "k").param("A", [1]).param("B", [2])
    with pytest.raises(kl.KLError) as e:
        d.restrict(bad)
    assert e.value.status == -1


def test_evaluation_errors():
    d = kl.KernelDef("x", "extern \"C\" __global__ void k() {}", "k").param("A", [3])
    for expr in ("problem_x / (A - A)", "A % 0", "A * 9223372036854775807", "div_ceil(A, 0)",
                 "unknown_name"):
        d.geometry(shared_memory=expr)
        with pytest.raises(kl.KLError):
            d.launch_geometry("default", (4,))


def test_definition_errors():
    with pytest.raises(kl.KLError):
        kl.KernelDef("not a name", VADD, "vadd")
    d = kl.KernelDef("v", VADD, "vadd")
    for name, values, default in [("BLOCK", [1, 1], 1), ("BLOCK", [1, 2], 3), ("problem_x", [1], 1),
                                  ("9x", [1], 1), ("BLOCK", [], 0)]:
        with pytest.raises(kl.KLError):
            d.param(name, values, default)
    d.param("BLOCK", [1])
    with pytest.raises(kl.KLError):
        d.param("BLOCK", [2])


def test_nvrtc_compiles_definitions():
    log = vadd_def().compile_only("BLOCK=128,ELEMS=4")
    assert "registers" in log and "symbol vadd" in log
    t = kl.KernelDef("scale3", SCALE, "scale<3>")
    log = t.compile_only()
    assert "symbol _Z5scaleILi3EEvPfi" in log
    # a parameter can reach the template through the options
    u = kl.KernelDef("scalep", SCALE, "scale<FACTOR>").param("FACTOR", [2, 4], 2)
    assert "symbol _Z5scaleILi4EEvPfi" in u.compile_only("FACTOR=4")
    bad = kl.KernelDef("bad", "extern \"C\" __global__ void k() { undefined_thing; }", "k")
    with pytest.raises(kl.KLError) as e:
        bad.compile_only()
    assert e.value.status == -3


def test_argument_marshalling():
    """kl_arg records from (kind, value) pairs: scalars point at their value
    with its size, buffers carry pointer, byte size, direction and dtype."""
    import ctypes
    import torch
    a = torch.zeros(10, dtype=torch.float32)
    b = torch.zeros(3, dtype=torch.float64)
    c = torch.zeros(6, dtype=torch.int32)
    d = torch.zeros(4, dtype=torch.bfloat16)
    e = torch.zeros(5, dtype=torch.int8)
    arr, keep = kl.make_args([("in", a), ("out", b), ("inout", c), ("in", d), ("out", e),
                              ("i32", -7), ("f64", 2.5), ("i64", 1 << 40)])
    got = [(x.ptr, x.bytes, x.kind, x.dtype) for x in arr]
    assert got[:5] == [(a.data_ptr(), 40, 1, 1), (b.data_ptr(), 24, 2, 0), (c.data_ptr(), 24, 3, 4),
                       (d.data_ptr(), 8, 1, 2), (e.data_ptr(), 5, 2, 5)]
    assert [x[1:] for x in got[5:]] == [(4, 0, 0), (8, 0, 0), (8, 0, 0)]
    assert ctypes.c_int32.from_address(got[5][0]).value == -7
    assert ctypes.c_double.from_address(got[6][0]).value == 2.5
    assert ctypes.c_int64.from_address(got[7][0]).value == 1 << 40
    with pytest.raises(ValueError):
        kl.make_args([("half", 1.0)])
