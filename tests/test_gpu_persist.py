"""Configuration and persisted selection state on the GPU: SR_VARIANT steers
the library's choice; the autotuner memo written through SR_TUNE_FILE is
reused by the next process; a selector saved to a file loads into one that
chooses identically; SR_MODEL_FILE serves calls made without a selector."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIMS = (9, 64, 40)


def _child(code, env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", textwrap.dedent(code)], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout.strip().splitlines()[-1]


# A child that sums 2^20 + 3 int32 ones through the given entry and prints the
# result, the resolved plan of the library's choice, and the memo size.
SUM_CHILD = """
    import torch, paper_2004_05371_gb300 as sr
    sr.load()
    n = (1 << 20) + 3
    x = torch.ones(n, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    before = sr.tune_size()
    if "{entry}" == "selected":
        st = sr.reduce_sum_selected_ptr(None, x.data_ptr(), n, sr.I32, out.data_ptr())
    else:
        st = sr.lib().sr_reduce_sum(sr.ctypes.c_void_p(x.data_ptr()), n, sr.I32,
                                    sr.ctypes.c_void_p(out.data_ptr()), 0, None)
    torch.cuda.synchronize()
    r = sr.Config()
    ps = sr.lib().sr_plan(n, sr.I32, None, sr.ctypes.byref(r))
    print(st, int(out.item()), ps, r.variant, before, sr.tune_size())
"""


@pytest.mark.parametrize("text", ["two_kernel", "grid_sync+bulk", "atomic", "0x403"])
def test_sr_variant_steers_the_library_choice(sr, text):
    want = sr.parse_variant(text)
    st, total, ps, variant, _, _ = (int(v) for v in _child(SUM_CHILD.format(entry="plain"),
                                                          {"SR_VARIANT": text}).split())
    assert st == sr.OK and ps == sr.OK
    assert total == (1 << 20) + 3
    assert variant & 0xF == want & 0xF
    assert bool(variant & sr.F_BULK) == bool(want & sr.F_BULK)


def test_tune_file_carries_the_autotuned_choice_to_the_next_process(sr, tmp_path):
    p = tmp_path / "tune.txt"
    env = {"SR_TUNE_FILE": str(p)}
    st, total, _, _, before, after = (int(v) for v in _child(SUM_CHILD.format(entry="selected"), env).split())
    assert st == sr.OK and total == (1 << 20) + 3
    assert (before, after) == (0, 1)
    text = p.read_text()
    lines = [l for l in text.splitlines() if l and not l.startswith("#")]
    assert lines[0] == "sr-tune 1" and lines[1].startswith("device ") and len(lines) == 3
    # the next process finds the entry at first use and tunes nothing
    st, total, _, _, before, after = (int(v) for v in _child(SUM_CHILD.format(entry="selected"), env).split())
    assert st == sr.OK and total == (1 << 20) + 3
    assert (before, after) == (1, 1)
    assert p.read_text() == text


def _selector(sr, seed=5):
    rng = np.random.default_rng(seed)
    m = sr.MLP(*DIMS)
    m.set_params(rng.normal(0, 0.3, m.P).astype(np.float32))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mu = rng.normal(0, 1, DIMS[0]).astype(np.float32)
    sd = rng.uniform(0.5, 2, DIMS[0]).astype(np.float32)
    return sr.NativeSelector(m, mu, sd, sr.candidates(sms))


SHAPES = [(1 << k, dt, nseg) for k in range(10, 31, 3) for dt in (0, 1, 2, 3) for nseg in (1, 100, 100000)]


def test_selector_file_round_trip(sr, tmp_path):
    s = _selector(sr)
    p = tmp_path / "sel.txt"
    s.save(str(p))
    t = sr.NativeSelector.load(str(p))
    for n, dt, nseg in SHAPES:
        mean = n / nseg
        a = s.choose(n, dt, nseg, mean, 0.5 * mean, 4 * mean).as_dict()
        b = t.choose(n, dt, nseg, mean, 0.5 * mean, 4 * mean).as_dict()
        assert a == b, (n, dt, nseg)
    q = tmp_path / "sel2.txt"
    t.save(str(q))
    assert q.read_text() == p.read_text()      # parameters, normalisation and candidates kept exactly
    t.close()
    s.close()


def test_selector_file_of_another_device_is_refused(sr, tmp_path):
    s = _selector(sr)
    p = tmp_path / "sel.txt"
    s.save(str(p))
    lines = p.read_text().splitlines(keepends=True)
    f = lines[1].split()
    assert f[0] == "device"
    lines[1] = " ".join(f[:2] + [str(int(f[2]) + 1)] + f[3:]) + "\n"   # another driver version
    q = tmp_path / "other.txt"
    q.write_text("".join(lines))
    h = sr.ctypes.c_void_p()
    assert sr.lib().sr_selector_load(str(q).encode(), sr.ctypes.byref(h)) == sr.ERR_UNSUPPORTED
    assert not h.value
    s.close()


def test_model_file_env_serves_calls_without_a_selector(sr, tmp_path):
    s = _selector(sr)
    p = tmp_path / "sel.txt"
    s.save(str(p))
    s.close()
    st, total, _, _, before, after = (int(v) for v in _child(SUM_CHILD.format(entry="selected"),
                                                           {"SR_MODEL_FILE": str(p)}).split())
    assert st == sr.OK and total == (1 << 20) + 3
    assert (before, after) == (0, 0)      # the selector chose: the autotuner never ran
    # a file that does not load: the calls return its status
    p.write_text("sr-selector 1\n")
    st = int(_child(SUM_CHILD.format(entry="selected"), {"SR_MODEL_FILE": str(p)}).split()[0])
    assert st == sr.ERR_ARG
