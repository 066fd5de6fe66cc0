"""The benchmark reads the DRAM traffic of its step kernel from a committed ncu
summary only while that summary was taken on the current kernel code.  These
tests pin the code hash it compares: comments and layout do not change it, any
code token does, and string literals that look like comments are code."""
import os
import re
import shutil

import bench


def test_strip_keeps_literals_and_drops_comments():
    src = ('int a = 1; // one\n'
           'const char* s = "x // y /* z */";  /* block\n comment */ char c = \'/\';\n'
           "char e = '\\''; int b = a / 2; const char* t = \"q\\\"//\";\n")
    out = bench.strip_c_comments(src)
    assert "one" not in out and "block" not in out and "comment" not in out
    assert '"x // y /* z */"' in out
    assert "'/'" in out and "'\\''" in out and "a / 2" in out
    assert '"q\\"//"' in out


def _copy_sources(tmp_path):
    csrc = os.path.join(bench.ROOT, "paper_1806_10589_gb300", "csrc")
    root = tmp_path / "repo"
    dst = root / "paper_1806_10589_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in bench.STEP_KERNEL_SOURCES:
        shutil.copy(os.path.join(csrc, f), dst / f)
    return root, dst


def _sha_at(root, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(root))
    return bench.kernel_sources_sha()


def test_hash_ignores_comments_and_layout_but_not_code(tmp_path, monkeypatch):
    root, dst = _copy_sources(tmp_path)
    base = _sha_at(root, monkeypatch)
    k = dst / "lbm_kernels.cu"
    src = k.read_text()
    # a new comment line and re-indented code: same hash
    k.write_text("// an added comment line\n" + src.replace("\n    ", "\n        ", 5))
    assert _sha_at(root, monkeypatch) == base
    # one changed constant in the code: a different hash
    m = re.search(r"#define LBM_AA_PREFETCH (\d+)", src)
    assert m, "the prefetch distance macro moved"
    k.write_text(src.replace(m.group(0), "#define LBM_AA_PREFETCH %d" % (int(m.group(1)) + 1)))
    assert _sha_at(root, monkeypatch) != base


def test_profile_traffic_only_for_the_profiled_code():
    sha = bench.kernel_sources_sha()
    for variant, path in bench.PROFILE_TRAFFIC.items():
        txt = open(path).read()
        m = re.search(r"kernel_sources_sha:\s*([0-9a-f]{16})", txt)
        assert m, path
        if m.group(1) == sha:
            assert bench.profiled_traffic(sha, variant) > 0
        else:  # code changed since the capture: no traffic figure
            assert bench.profiled_traffic(sha, variant) is None
        assert bench.profiled_traffic("0" * 16, variant) is None
