"""Host-side logic of libkl, no GPU needed: the library loads and exports
every symbol of include/kl.h, the configuration space of Table 2, config
parsing and constraints, run-time compilation with NVRTC for sm_103a, the
wisdom-selection heuristic of Sec. 4.5, and the recommended layout."""

from __future__ import annotations

import os
import re

import pytest

from paper_2303_12374_gb300 import kl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    text = open(os.path.join(ROOT, "include", "kl.h")).read()
    return sorted(set(re.findall(r"\b(kl_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = kl.load()
    names = header_symbols()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(kl.SIGNATURES), set(names) ^ set(kl.SIGNATURES)
    assert "sm_103a" in kl.kl_version()


def _golden_space():
    vals = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "table2_space.txt")):
        line = line.strip()
        if not line or line.startswith("#") or line.startswith("default"):
            continue
        name, *rest = line.split()
        vals[name] = rest
    return vals


def test_space_is_table2():
    vals = _golden_space()
    count = 1
    for name, v in vals.items():
        if name != "more_than":
            count *= len(v)
    op = kl.Op(5, 1, 1, 0)
    assert kl.kl_space_size(op, 0) == count
    assert count > int(vals["more_than"][0])
    # every raw index decodes to values of the table
    seen = {k: set() for k in ("bx", "by", "bz", "tx", "perm", "minb")}
    for idx in range(0, count, 997):
        text, _ = kl.kl_space_config(op, 0, idx)
        kv = dict(item.split("=") for item in text.split(":", 1)[1].split(","))
        for k in seen:
            seen[k].add(kv[k])
    assert seen["bx"] == set(vals["block_size_x"])
    assert seen["by"] == set(vals["block_size_y"]) == seen["bz"]
    assert seen["tx"] == set(vals["tile_factor_x"])
    assert seen["perm"] == set(vals["unravel"])
    assert seen["minb"] == set(vals["min_blocks_per_sm"])


def test_default_config_is_table2_default():
    op = kl.Op(5, 1, 1, 0)
    d = kl.kl_config_normalize(op, "default")
    assert d == ("direct:bx=256,by=1,bz=1,tx=1,ty=1,tz=1,ux=0,uy=0,uz=0,cx=0,cy=0,cz=0,"
                 "perm=XYZ,minb=1")
    assert kl.kl_config_normalize(op, "direct:bx=32,perm=ZYX") .startswith("direct:bx=32,")


@pytest.mark.parametrize("bad", ["direct:bx=512", "direct:bx=256,by=8",  # > 1024 threads
                                 "direct:tx=3", "direct:perm=ABC", "direct:minb=7",
                                 "direct:foo=1", "nosuch:bx=1", "direct:bx",
                                 "zpack:w=4,ly=2,cs=1,yx=1",       # cs forms its own y faces
                                 "zpack:w=16,ly=1,cs=1",           # 1536 threads per block
                                 "zpack:w=8,ly=1,cs=1,minb=3",     # 2304 threads per SM
                                 "zpack:w=4,ly=2,cs=2"])
def test_invalid_configs_are_rejected(bad):
    with pytest.raises(kl.KLError) as e:
        kl.kl_config_normalize(kl.Op(5, 1, 1, 0), bad)
    assert e.value.status == -1


@pytest.mark.parametrize("dtype", [0, 1, 2, 3])
@pytest.mark.parametrize("adv,diff", [(5, 1), (2, 2), (0, 1), (5, 0)])
def test_nvrtc_compiles_for_sm103a(dtype, adv, diff):
    log = kl.kl_compile_only(kl.Op(adv, diff, dtype, 0), "default", 1, 0)
    assert "sm_103a" in log and "registers" in log
    assert "spill stores" in log


def test_nvrtc_compiles_tiled_configs():
    op = kl.Op(5, 2, 1, 1)
    for cfg in ["direct:bx=32,by=4,bz=2,tx=2,tz=2,ux=1,uz=1,cx=1,cz=1,perm=ZXY,minb=2",
                "direct:bx=64,by=2,tx=4,ty=2,ux=1,uy=1,cx=1,perm=YZX"]:
        log = kl.kl_compile_only(op, cfg, 0, 1)
        m = re.search(r"(\d+) bytes spill stores", log)
        assert m is not None
    # zpack, all components per thread and one warp group per component
    for cfg in ["zpack:w=4,ly=2,kc=16,ns=8,minb=2", "zpack:w=4,ly=2,kc=16,ns=8,minb=2,cs=1"]:
        log = kl.kl_compile_only(kl.Op(5, 1, 1, 0), cfg, 1, 1)
        assert re.search(r"(\d+) bytes spill stores", log) is not None
    # zpack with variable nu (stretched z)
    log = kl.kl_compile_only(kl.Op(5, 2, 1, 0), "zpack:w=4,ly=2,kc=16,ns=8,minb=2", 1, 0)
    assert re.search(r"(\d+) bytes spill stores", log) is not None


def test_out_f32_only_with_16bit_storage():
    for dt in (0, 1):
        with pytest.raises(kl.KLError) as e:
            kl.kl_compile_only(kl.Op(5, 1, dt, 0, 1), "default", 1, 1)
        assert "16-bit" in str(e.value)
    log = kl.kl_compile_only(kl.Op(5, 1, 2, 0, 1), "zpack:w=4,ly=2,kc=16,ns=8,minb=2", 1, 1)
    assert "registers" in log


def test_zpack_variable_nu_needs_cs0_yx0():
    for bad in ("zpack:w=4,ly=2,cs=1", "zpack:w=4,ly=2,yx=1"):
        with pytest.raises(kl.KLError):
            kl.kl_config_normalize(kl.Op(5, 2, 1, 0), bad)
    assert kl.kl_config_normalize(kl.Op(5, 2, 1, 0), "zpack:w=4,ly=2").startswith("zpack:")


def test_nvrtc_failure_is_reported():
    # a configuration the space accepts but the zmarch family rejects at compile
    # time is not reachable; an invalid define is reported as INVALID_ARG first
    with pytest.raises(kl.KLError) as e:
        kl.kl_compile_only(kl.Op(5, 1, 1, 0), "direct:bx=7", 0, 1)
    assert e.value.status == -1


# ------------------------------------------------------------- wisdom

def _write(path, lines):
    with open(path, "w") as f:
        f.write("# test wisdom\n")
        for l in lines:
            f.write(l + "\n")


def rec(dev, cc, zbc, n, cfg):
    return (f'device="{dev}" cc={cc} zbc={zbc} nx={n[0]} ny={n[1]} nz={n[2]} '
            f'config="{cfg}" time_us=1.0 date=2026-01-01')


def test_wisdom_rules(tmp_path):
    p = str(tmp_path / "w.wisdom")
    _write(p, [
        rec("GPU A", "10.3", 1, (256, 256, 256), "direct:bx=32"),
        rec("GPU A", "10.3", 1, (512, 512, 256), "direct:bx=64"),
        rec("GPU B", "10.3", 1, (128, 128, 128), "direct:bx=128"),
        rec("GPU C", "9.0", 1, (64, 64, 64), "direct:bx=16"),
        rec("GPU A", "10.3", 0, (256, 256, 256), "direct:by=2"),
        rec("GPU A", "10.3", 1, (256, 256, 256), "direct:bx=32,by=2"),  # newer duplicate
    ])
    sel = lambda dev, cc, zbc, n: kl.kl_wisdom_select(p, dev, cc[0], cc[1], zbc, *n)
    # rule 1, equal times: the newest duplicate wins
    assert sel("GPU A", (10, 3), 1, (256, 256, 256)) == ("direct:bx=32,by=2", 1)
    # rule 2: same device, nearest size
    assert sel("GPU A", (10, 3), 1, (500, 500, 250)) == ("direct:bx=64", 2)
    # ... where the nearest size has two sessions, they compete as in rule 1
    assert sel("GPU A", (10, 3), 1, (300, 300, 300)) == ("direct:bx=32,by=2", 2)
    # zbc never crosses
    assert sel("GPU A", (10, 3), 0, (512, 512, 256)) == ("direct:by=2", 2)
    # rule 3: other device, same architecture, nearest size
    assert sel("GPU Z", (10, 3), 1, (100, 100, 100)) == ("direct:bx=128", 3)
    # rule 4: other architecture, nearest size of any record
    assert sel("GPU Z", (12, 0), 1, (60, 60, 60)) == ("direct:bx=16", 4)
    # rule 5: nothing for this zbc ... and a missing file
    assert sel("GPU Z", (12, 0), 2, (60, 60, 60)) == ("default", 5)
    assert kl.kl_wisdom_select(str(tmp_path / "none"), "x", 1, 0, 0, 1, 1, 1) == ("default", 5)


def test_wisdom_duplicates_fastest_session_wins(tmp_path):
    p = str(tmp_path / "w.wisdom")
    _write(p, [rec("G", "10.3", 0, (64, 64, 64), "direct:bx=16").replace("time_us=1.0", "time_us=9.0"),
               rec("G", "10.3", 0, (64, 64, 64), "direct:bx=32").replace("time_us=1.0", "time_us=3.0"),
               rec("G", "10.3", 0, (64, 64, 64), "direct:bx=64").replace("time_us=1.0", "time_us=5.0")])
    assert kl.kl_wisdom_select(p, "G", 10, 3, 0, 64, 64, 64) == ("direct:bx=32", 1)


def test_wisdom_nearest_size_takes_its_fastest_session(tmp_path):
    p = str(tmp_path / "w.wisdom")
    _write(p, [rec("G", "10.3", 0, (64, 64, 64), "direct:bx=16").replace("time_us=1.0", "time_us=9.0"),
               rec("G", "10.3", 0, (256, 256, 256), "direct:bx=128"),
               rec("G", "10.3", 0, (64, 64, 64), "direct:bx=32").replace("time_us=1.0", "time_us=3.0"),
               rec("G", "10.3", 0, (64, 64, 64), "direct:bx=64").replace("time_us=1.0", "time_us=5.0")])
    assert kl.kl_wisdom_select(p, "G", 10, 3, 0, 70, 60, 64) == ("direct:bx=32", 2)


def test_batch_selection_by_total_points(tmp_path):
    """A batch takes the record whose tuned problem has the point count
    nearest (in ratio) to the batch's total: 64 grids of ~1 M points go to the
    512 x 512 x 256 record, not to the small grids' records; the device and
    zbc tiers and the fastest session of a size apply as for one grid."""
    p = str(tmp_path / "w.wisdom")
    _write(p, [
        rec("G", "10.3", 1, (64, 64, 64), "zpack:w=4,ly=1"),
        rec("G", "10.3", 1, (256, 256, 256), "zpack:w=4,ly=3"),
        rec("G", "10.3", 1, (512, 512, 256), "zpack:w=8,ly=4").replace("time_us=1.0", "time_us=9.0"),
        rec("G", "10.3", 1, (512, 512, 256), "zpack:w=8,ly=3").replace("time_us=1.0", "time_us=5.0"),
        rec("G", "10.3", 0, (64, 64, 64), "zpack:w=2,ly=2"),
        rec("H", "10.3", 1, (1024, 1024, 1024), "zpack:w=16,ly=2"),
    ])
    sel = lambda dev, zbc, n: kl.kl_wisdom_select_points(p, dev, 10, 3, zbc, n)
    assert sel("G", 1, 64 * 1_100_000) == ("zpack:w=8,ly=3", 2)      # fastest 512x512x256 session
    assert sel("G", 1, 300_000) == ("zpack:w=4,ly=1", 2)            # 262 144 points
    assert sel("G", 1, 10_000_000) == ("zpack:w=4,ly=3", 2)         # ln ratio 0.52 vs 1.90
    assert sel("G", 0, 10 ** 9) == ("zpack:w=2,ly=2", 2)            # zbc never crosses
    assert sel("X", 1, 10 ** 9) == ("zpack:w=16,ly=2", 3)           # same architecture
    assert kl.kl_wisdom_select_points(str(tmp_path / "none"), "G", 10, 3, 1, 5) == ("default", 5)


def test_wisdom_distance_tie_takes_first_record(tmp_path):
    p = str(tmp_path / "w.wisdom")
    _write(p, [rec("G", "10.3", 0, (100, 100, 100), "direct:bx=16"),
               rec("G", "10.3", 0, (300, 100, 100), "direct:bx=32")])
    assert kl.kl_wisdom_select(p, "G", 10, 3, 0, 200, 100, 100) == ("direct:bx=16", 2)


def test_corrupt_wisdom_falls_back_to_default(tmp_path):
    p = str(tmp_path / "w.wisdom")
    _write(p, ['device="G" cc=10.3 nx=1 ny=2'])   # no nz / config
    assert kl.kl_wisdom_select(p, "G", 10, 3, 0, 1, 2, 3) == ("default", 5)
    assert "record lacks" in kl.last_error()


def test_wisdom_append_round_trip(tmp_path):
    p = str(tmp_path / "w.wisdom")
    kl.kl_wisdom_append(p, "NVIDIA GB300", 10, 3, 1, 256, 256, 256, "direct:bx=64", 61.5,
                        "strategy=random evals=10")
    kl.kl_wisdom_append(p, "NVIDIA GB300", 10, 3, 1, 512, 512, 256, "direct:bx=32", 200.0, "")
    text = open(p).read()
    assert text.count("\n") == 3 and "strategy=random" in text
    assert kl.kl_wisdom_select(p, "NVIDIA GB300", 10, 3, 1, 256, 256, 256) == ("direct:bx=64", 1)


# ------------------------------------------------------------- layout

@pytest.mark.parametrize("dtype,es", [(0, 8), (1, 4), (2, 2), (3, 2)])
def test_layout_alignment(dtype, es):
    sj, sk, origin, extent = kl.kl_layout(256, 200, 64, 3, dtype)
    x0 = origin % sj
    assert (x0 * es) % 128 == 0 and (sj * es) % 128 == 0
    assert x0 >= 3 and x0 + 256 + 3 <= sj
    assert sk == sj * 206 and extent == sk * 70
    assert origin == x0 + 3 * sj + 3 * sk


def test_layout_rejects_huge():
    with pytest.raises(kl.KLError):
        kl.kl_layout(4096, 4096, 200, 3, 0)


# ------------------------------------------------------------- cubin cache

def _cubins(d):
    return sorted(p for p in os.listdir(d) if p.endswith(".cubin"))


def test_cache_prepare_writes_once_and_reuses(tmp_path):
    d = str(tmp_path)
    op = kl.Op(5, 1, 1, 0)
    cfg = "zpack:w=4,ly=2,kc=16,ns=8,minb=1"
    assert kl.kl_cache_prepare(d, op, cfg, 1, 1) is False
    files = _cubins(d)
    assert len(files) == 1 and files[0].startswith("kl_")
    assert kl.kl_cache_prepare(d, op, cfg, 1, 1) is True
    # the same configuration text in another spelling is the same variant
    assert kl.kl_cache_prepare(d, op, kl.kl_config_normalize(op, cfg), 1, 1) is True
    # anything that changes the compile defines is another file
    assert kl.kl_cache_prepare(d, op, cfg, 0, 1) is False
    assert kl.kl_cache_prepare(d, op, "batch+" + cfg, 1, 1) is False
    assert kl.kl_cache_prepare(d, kl.Op(5, 1, 0, 0), "default", 1, 1) is False
    assert len(_cubins(d)) == 4
    assert not [p for p in os.listdir(d) if p.endswith(".tmp")]
    head = open(os.path.join(d, files[0]), "rb").readline().decode()
    assert head.startswith("KLCUBIN1 ")


def test_cache_rejects_damaged_or_foreign_files(tmp_path):
    d = str(tmp_path)
    op = kl.Op(5, 1, 1, 0)
    kl.kl_cache_prepare(d, op, "default", 1, 1)
    (f,) = _cubins(d)
    path = os.path.join(d, f)
    good = open(path, "rb").read()
    # a flipped byte in the cubin fails the checksum: recompiled and rewritten
    bad = bytearray(good)
    bad[-100] ^= 0x5A
    open(path, "wb").write(bytes(bad))
    assert kl.kl_cache_prepare(d, op, "default", 1, 1) is False
    assert open(path, "rb").read() == good
    # truncated, and with trailing bytes
    open(path, "wb").write(good[:-10])
    assert kl.kl_cache_prepare(d, op, "default", 1, 1) is False
    open(path, "wb").write(good + b"x")
    assert kl.kl_cache_prepare(d, op, "default", 1, 1) is False
    # another variant's file under this name (identity mismatch)
    kl.kl_cache_prepare(d, op, "direct:bx=64", 1, 1)
    other = [p for p in _cubins(d) if p != f][0]
    open(path, "wb").write(open(os.path.join(d, other), "rb").read())
    assert kl.kl_cache_prepare(d, op, "default", 1, 1) is False
    assert kl.kl_cache_prepare(d, op, "default", 1, 1) is True


def test_cache_argument_errors(tmp_path):
    op = kl.Op(5, 1, 1, 0)
    with pytest.raises(kl.KLError) as e:
        kl.kl_cache_prepare(str(tmp_path / "missing"), op, "default", 1, 1)
    assert e.value.status == -4
    with pytest.raises(kl.KLError) as e:
        kl.kl_cache_prepare(str(tmp_path), op, "direct:bx=7", 1, 1)
    assert e.value.status == -1
    with pytest.raises(kl.KLError) as e:
        kl.kl_set_cache_dir(None, str(tmp_path))
    assert e.value.status == -1


def test_c_abi_from_plain_c(tmp_path):
    """The boundary is a C ABI: a C program built with gcc against include/kl.h
    and linked to libkl.so calls the host-only entry points."""
    import subprocess
    from paper_2303_12374_gb300 import build as kbuild
    lib = kbuild.build()
    exe = str(tmp_path / "abi_host")
    subprocess.check_call(["gcc", "-std=c11", "-O1", "-Wall", "-Werror",
                           "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c", "abi_host.c"), "-o", exe,
                           "-L", os.path.dirname(lib), "-lkl", "-lm",
                           "-Wl,-rpath," + os.path.dirname(lib)])
    r = subprocess.run([exe, str(tmp_path)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("all ok")


def test_copy_in_out_reject_bad_arguments_before_any_cuda_call():
    grid = kl.Grid(8, 8, 8, 1, 10, 100, 111, 1000, 1, 0, 0.125, 0.125, 0.125, 1e-3, None)
    with pytest.raises(kl.KLError):
        kl.kl_copy_in(1, grid, None, 1, None)
    with pytest.raises(kl.KLError):
        kl.kl_copy_out(7, grid, 1, 1, None)
    bad = kl.Grid(8, 8, 8, 1, 4, 100, 111, 1000, 1, 0, 0.125, 0.125, 0.125, 1e-3, None)
    with pytest.raises(kl.KLError):                # sj smaller than a padded row
        kl.kl_copy_in(1, bad, 1, 1, None)
