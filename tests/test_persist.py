"""Configuration and persisted selection state on the host: SR_VARIANT's
syntax, the autotuner memo's file format (save, load, merge, refusal of
malformed files, SR_TUNE_FILE at first use) and the selector file's parser.
No GPU needed: none of these paths makes a device call before its file
parses."""
import os
import subprocess
import sys
import textwrap

import pytest

import paper_2004_05371_gb300 as sr
from paper_2004_05371_gb300 import build as sr_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    sr_build.build()
    return sr.load()


@pytest.fixture
def clean_memo(lib):
    sr.tune_clear()
    yield
    sr.tune_clear()


@pytest.mark.parametrize("text,want", [
    ("0", 0), ("3", 3), ("0x403", 0x403), (" 1027 \n", 1027),
    ("auto", sr.AUTO), ("two_kernel", sr.TWO_KERNEL), ("atomic", sr.ATOMIC), ("last_block", sr.LAST_BLOCK),
    ("grid_sync", sr.GRID_SYNC), ("single_cluster", 5),
    ("last_block+bulk", sr.LAST_BLOCK | sr.F_BULK),
    ("two_kernel+cluster4+kahan", sr.TWO_KERNEL | sr.CLUSTER(2) | sr.F_KAHAN),
    ("grid_sync+fp64_combine", sr.GRID_SYNC | sr.F_FP64_COMBINE),
    ("kahan+fp64_auto", sr.F_KAHAN | 0x1000), ("cluster16", sr.CLUSTER(4)), ("bulk", sr.F_BULK),
])
def test_parse_variant(lib, text, want):
    assert sr.parse_variant(text) == want


@pytest.mark.parametrize("text", ["", "  ", "foo", "3junk", "-1", "0x", "atomic+last_block", "kahan+kahan",
                                  "cluster2+cluster4", "last_block+", "+bulk", "LAST_BLOCK", "99999999999"])
def test_parse_variant_rejects(lib, text):
    v = sr.ctypes.c_int(-7)
    assert lib.sr_parse_variant(text.encode(), sr.ctypes.byref(v)) == sr.ERR_ARG
    assert v.value == -7  # untouched


TABLE = textwrap.dedent("""\
    sr-tune 1
    # a comment line
    device 152 13000 NVIDIA GB300
    e 268435456 0 1 453 0 453 3 160 0 0 16 4 0 0 1
    e 4096 1 1 192 0 192 5 128 0 0 16 2 0 0 1
    device 132 12090 NVIDIA H100 80GB HBM3
    e 1048576 2 1000 107 0 107 1027 288 1 0 16 4 65536 2 0.5
    """)


def _entries(text):
    """(device, entry) pairs of a table, comments dropped."""
    dev, out = None, set()
    for line in text.splitlines():
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "device":
            dev = " ".join(f[1:])
        elif f[0] == "e":
            out.add((dev, " ".join(f[1:])))
    return out


def test_tune_table_round_trip(clean_memo, tmp_path):
    src = tmp_path / "in.txt"
    src.write_text(TABLE)
    assert sr.tune_load(str(src)) == 3
    assert sr.tune_size() == 3
    dst = tmp_path / "out.txt"
    sr.tune_save(str(dst))
    text = dst.read_text()
    assert text.startswith("sr-tune 1\n")
    assert _entries(text) == _entries(TABLE)
    # loading the saved file again replaces equal keys: still three entries
    assert sr.tune_load(str(dst)) == 3
    assert sr.tune_size() == 3
    sr.tune_clear()
    assert sr.tune_size() == 0
    assert sr.tune_load(str(dst)) == 3 and sr.tune_size() == 3


def test_tune_load_merges_and_replaces(clean_memo, tmp_path):
    a = tmp_path / "a.txt"
    a.write_text(TABLE)
    b = tmp_path / "b.txt"
    # the same key as the first entry, another configuration; and one new entry
    b.write_text("sr-tune 1\ndevice 152 13000 NVIDIA GB300\n"
                 "e 268435456 0 1 453 0 453 1 512 8 0 32 2 0 0 1\n"
                 "e 1024 0 1 160 0 160 5 32 0 0 16 2 0 0 1\n")
    sr.tune_load(str(a))
    assert sr.tune_load(str(b)) == 2
    assert sr.tune_size() == 4
    out = tmp_path / "merged.txt"
    sr.tune_save(str(out))
    got = _entries(out.read_text())
    assert ("152 13000 NVIDIA GB300", "268435456 0 1 453 0 453 1 512 8 0 32 2 0 0 1") in got
    assert ("152 13000 NVIDIA GB300", "268435456 0 1 453 0 453 3 160 0 0 16 4 0 0 1") not in got


@pytest.mark.parametrize("bad", [
    "",                                                    # no header
    "sr-tune 2\n",                                         # unknown version
    "sr-tune\n",                                           # no version
    "sr-tune 1\ne 1 0 1 0 0 0 3 0 0 0 16 4 0 0 1\n",       # entry before any device line
    "sr-tune 1\ndevice 152 13000\n",                      # device line without a name
    "sr-tune 1\ndevice x 13000 GB300\n",                  # non-numeric SM count
    "sr-tune 1\ndevice 152 13000 GB300\ne 1 0 1 0 0 0 3 0 0 0 16 4 0 0\n",      # short entry
    "sr-tune 1\ndevice 152 13000 GB300\ne 1 9 1 0 0 0 3 0 0 0 16 4 0 0 1\n",    # bad dtype
    "sr-tune 1\ndevice 152 13000 GB300\ne 1 0 0 0 0 0 3 0 0 0 16 4 0 0 1\n",    # nseg 0
    "sr-tune 1\ndevice 152 13000 GB300\ne 1 0 1 0 0 0 3 -5 0 0 16 4 0 0 1\n",   # negative field
    "sr-tune 1\ndevice 152 13000 GB300\ne 1 0 1 0 0 0 3 0 0 0 16 4 0 0 nan\n",  # NaN scale
    "sr-tune 1\ndevice 152 13000 GB300\nx 1 0 1 0 0 0 3 0 0 0 16 4 0 0 1\n",    # unknown line
])
def test_tune_load_rejects_malformed_and_changes_nothing(clean_memo, tmp_path, bad):
    good = tmp_path / "good.txt"
    good.write_text(TABLE)
    sr.tune_load(str(good))
    p = tmp_path / "bad.txt"
    # a good entry before the bad line where there is a device section: a file
    # that fails anywhere must merge nothing
    lines = bad.splitlines(keepends=True)
    for i, line in enumerate(lines):
        if line.startswith("device ") and len(line.split()) >= 4:
            lines.insert(i + 1, "e 7 0 1 0 0 0 3 0 0 0 16 4 0 0 1\n")
            break
    p.write_text("".join(lines))
    k = sr.ctypes.c_int64(-1)
    assert sr.lib().sr_tune_load(str(p).encode(), sr.ctypes.byref(k)) == sr.ERR_ARG
    assert sr.tune_size() == 3


def test_tune_paths_rejected(clean_memo, tmp_path):
    L = sr.lib()
    assert L.sr_tune_load(None, None) == sr.ERR_ARG
    assert L.sr_tune_load(b"", None) == sr.ERR_ARG
    assert L.sr_tune_load(str(tmp_path / "missing.txt").encode(), None) == sr.ERR_ARG
    assert L.sr_tune_save(None) == sr.ERR_ARG
    assert L.sr_tune_save(str(tmp_path / "no" / "such" / "dir.txt").encode()) == sr.ERR_ARG


def _child(code, env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    return r.stdout.strip()


def test_tune_file_env_read_at_first_use(lib, tmp_path):
    p = tmp_path / "tune.txt"
    p.write_text(TABLE)
    out = _child("import paper_2004_05371_gb300 as sr; print(sr.tune_size())", {"SR_TUNE_FILE": str(p)})
    assert out == "3"
    # a malformed file is not used, and a save elsewhere leaves it as it was
    p.write_text("sr-tune 1\ngarbage\n")
    out = _child("import paper_2004_05371_gb300 as sr; print(sr.tune_size())", {"SR_TUNE_FILE": str(p)})
    assert out == "0"
    assert p.read_text() == "sr-tune 1\ngarbage\n"
    # a missing file: an empty memo until the first tuned call creates it
    q = tmp_path / "new.txt"
    out = _child("import paper_2004_05371_gb300 as sr; print(sr.tune_size())", {"SR_TUNE_FILE": str(q)})
    assert out == "0" and not q.exists()


def test_sr_variant_env_parse_failure_refuses_library_choice(lib):
    code = textwrap.dedent("""\
        import paper_2004_05371_gb300 as sr
        L = sr.lib()
        r = sr.Config()
        print(L.sr_plan(1 << 20, sr.F32, None, sr.ctypes.byref(r)),
              L.sr_plan(1 << 20, sr.F32, sr.ctypes.byref(sr.make_config(sr.LAST_BLOCK)), sr.ctypes.byref(r)),
              L.sr_reduce_sum(sr.ctypes.c_void_p(1 << 20), 1 << 20, sr.F32, sr.ctypes.c_void_p(1 << 20), 0, None))
        """)
    st = [int(v) for v in _child(code, {"SR_VARIANT": "last_block+nonsense"}).split()]
    assert st[0] == sr.ERR_ARG      # cfg NULL: the library's choice cannot be made
    assert st[1] != sr.ERR_ARG      # an explicit configuration ignores SR_VARIANT
    assert st[2] == sr.ERR_ARG      # variant SR_AUTO through sr_reduce_sum


SELECTOR = textwrap.dedent("""\
    sr-selector 1
    device 7 1 test device
    dims 9 2 2
    mu 0 0 0 0 0 0 0 0 0
    sd 1 1 1 1 1 1 1 1 1
    cands 2
    c 3 256 0 0 16 4 0 0 1
    c 1 256 0 0 16 4 0 0 1
    params 32
    """) + " ".join(["0.25"] * 32) + "\n"


@pytest.mark.parametrize("mutate", [
    lambda t: t.replace("sr-selector 1", "sr-selector 9"),
    lambda t: t.replace("dims 9 2 2", "dims 8 2 2"),
    lambda t: t.replace("cands 2", "cands 3"),
    lambda t: t.replace("params 32", "params 33"),
    lambda t: t.replace("params 32", "params 31"),
    lambda t: t.replace("mu 0 0", "mu 0 x"),
    lambda t: t.replace("c 1 256", "c 1 -256"),
    lambda t: t + "trailing\n",
    lambda t: "",
])
def test_selector_file_rejects_malformed_before_any_device_call(lib, tmp_path, mutate):
    p = tmp_path / "sel.txt"
    p.write_text(mutate(SELECTOR))
    h = sr.ctypes.c_void_p(123)
    assert lib.sr_selector_load(str(p).encode(), sr.ctypes.byref(h)) == sr.ERR_ARG
    assert not h.value


def test_selector_file_well_formed_reaches_the_device_check(lib, tmp_path):
    p = tmp_path / "sel.txt"
    p.write_text(SELECTOR)
    h = sr.ctypes.c_void_p()
    st = lib.sr_selector_load(str(p).encode(), sr.ctypes.byref(h))
    # no GPU here: the device query fails; on a GPU the identity check refuses
    # the file, stamped with a device of 7 SMs
    assert st in (sr.ERR_CUDA, sr.ERR_UNSUPPORTED)
    assert not h.value
    assert lib.sr_selector_load(str(tmp_path / "missing").encode(), sr.ctypes.byref(h)) == sr.ERR_ARG
    assert lib.sr_selector_load(str(p).encode(), None) == sr.ERR_ARG


def test_concurrent_saves_leave_one_whole_file(clean_memo, tmp_path):
    """Writers racing on one path (threads here; processes alike) each write a
    temporary file of their own and rename it: the survivor parses whole and
    no temporary file is left behind."""
    import concurrent.futures as cf
    src = tmp_path / "in.txt"
    src.write_text(TABLE)
    sr.tune_load(str(src))
    dst = tmp_path / "shared.txt"
    with cf.ThreadPoolExecutor(8) as ex:
        sts = list(ex.map(lambda _: sr.lib().sr_tune_save(str(dst).encode()), range(64)))
    assert all(st == sr.OK for st in sts)
    assert _entries(dst.read_text()) == _entries(TABLE)
    assert sorted(p.name for p in tmp_path.iterdir()) == ["in.txt", "shared.txt"]
