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
