"""The C ABI library loads and exports every symbol include/*.h declares;
host-only entry points behave without a GPU."""
import glob
import os
import re

import pytest

from paper_2603_15023_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(pac_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    L = B.lib()
    declared = _declared()
    assert {"pac_create", "pac_hash_keys", "pac_aggregate", "pac_finalize"} <= declared
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing
    assert set(B.EXPORTED) == declared


def test_query_key_matches_oracle():
    import oracle
    for seed in (0, 1, 2**63, 123456789):
        assert B.pac_query_key(seed) == oracle.query_key(seed)


def test_status_strings():
    assert B.status_name(B.PAC_E_OVERFLOW) == "PAC_E_OVERFLOW"
    assert B.status_name(B.PAC_OK) == "PAC_OK"


def test_null_context_is_rejected():
    L = B.lib()
    assert L.pac_hash_keys(None, None, None, 0, 0, 0, None) == B.PAC_E_INVALID
    assert L.pac_sync_status(None, None) == B.PAC_E_INVALID
    assert L.pac_create(None, 0) == B.PAC_E_INVALID


def test_create_without_gpu_fails_cleanly():
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a GPU is present")
    with pytest.raises(B.PacError):
        B.pac_create(0)


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of pac_input / pac_agg_spec / pac_query / pac_select_spec have the C
    header's sizes and field offsets (checked by compiling a probe with gcc)."""
    import ctypes
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "pac.h"\n'
        'int main(void) {\n'
        '  printf("%zu %zu %zu\\n", sizeof(pac_input), offsetof(pac_input, n_groups), offsetof(pac_input, n));\n'
        '  printf("%zu %zu %zu\\n", sizeof(pac_agg_spec), offsetof(pac_agg_spec, values), offsetof(pac_agg_spec, out));\n'
        '  printf("%zu %zu %zu %zu\\n", sizeof(pac_query), offsetof(pac_query, specs), offsetof(pac_query, seed),'
        ' offsetof(pac_query, flags));\n'
        '  printf("%zu %zu %zu %zu\\n", sizeof(pac_select_spec), offsetof(pac_select_spec, thr),'
        ' offsetof(pac_select_spec, n_thr), offsetof(pac_select_spec, thr_ids));\n'
        '  return 0;\n}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)])
    got = [list(map(int, line.split())) for line in subprocess.check_output([str(exe)], text=True).splitlines()]
    assert got[0] == [ctypes.sizeof(B.PacInput), B.PacInput.n_groups.offset, B.PacInput.n.offset]
    assert got[1] == [ctypes.sizeof(B.PacAggSpec), B.PacAggSpec.values.offset, B.PacAggSpec.out.offset]
    assert got[2] == [ctypes.sizeof(B.PacQuery), B.PacQuery.specs.offset, B.PacQuery.seed.offset,
                      B.PacQuery.flags.offset]
    assert got[3] == [ctypes.sizeof(B.PacSelectSpec), B.PacSelectSpec.thr.offset, B.PacSelectSpec.n_thr.offset,
                      B.PacSelectSpec.thr_ids.offset]
