"""The autotuner's tuning table (host logic, no GPU): JSON save and load, key buckets,
and rejection of malformed entries."""
import json

import pytest

from paper_2106_15319_gb300 import capi


@pytest.fixture(autouse=True)
def _clean_table():
    capi.load()
    capi.serial_emd_tune_clear()
    yield
    capi.serial_emd_tune_clear()


def _entry(**kw):
    e = dict(precision=capi.FP32_MIXED, stop=capi.STOP_FIXED, ensemble=0, batch_log2=0,
             len_log2=16, tile=512, ctas_per_sm=2, ms=1.25)
    e.update(kw)
    return e


def test_load_lookup_and_buckets(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"format": "serial_emd tuning table 1",
                                "entries": [_entry(), _entry(ensemble=1, batch_log2=8,
                                                             len_log2=18, tile=128,
                                                             ctas_per_sm=0)]}))
    capi.serial_emd_tune_load(str(path))
    p = capi.serial_emd_default_params(rows=256, cols=256)
    # L = 65536 is bucket 16; 40000 rounds up to 2^16 as well; 65537 does not
    assert capi.serial_emd_tune_lookup(p, 65536, 1) == (512, 2, 0)
    assert capi.serial_emd_tune_lookup(p, 40000, 1) == (512, 2, 0)
    assert capi.serial_emd_tune_lookup(p, 65537, 1) is None
    assert capi.serial_emd_tune_lookup(p, 65536, 2) is None
    p64 = capi.serial_emd_default_params(rows=256, cols=256, precision=capi.FP64)
    assert capi.serial_emd_tune_lookup(p64, 65536, 1) is None
    psd = capi.serial_emd_default_params(rows=256, cols=256, stop=capi.STOP_SD)
    assert capi.serial_emd_tune_lookup(psd, 65536, 1) is None
    pe = capi.serial_emd_default_params(rows=512, cols=512, ensemble_trials=256)
    assert capi.serial_emd_tune_lookup(pe, 262144, 256) == (128, 0, 0)


def test_save_round_trip(tmp_path):
    src = tmp_path / "a.json"
    src.write_text(json.dumps({"entries": [_entry(), _entry(len_log2=12, tile=256,
                                                            ctas_per_sm=0, variant=1,
                                                            ms=0.5)]}))
    capi.serial_emd_tune_load(str(src))
    out = tmp_path / "b.json"
    capi.serial_emd_tune_save(str(out))
    doc = json.loads(out.read_text())
    got = sorted((e["len_log2"], e["tile"], e["ctas_per_sm"], e["variant"])
                 for e in doc["entries"])
    assert got == [(12, 256, 0, 1), (16, 512, 2, 0)]
    capi.serial_emd_tune_clear()
    p = capi.serial_emd_default_params(rows=64, cols=64)
    assert capi.serial_emd_tune_lookup(p, 4096, 1) is None
    capi.serial_emd_tune_load(str(out))
    assert capi.serial_emd_tune_lookup(p, 4096, 1) == (256, 0, 1)


def test_malformed_entries_are_skipped_and_bad_files_rejected(tmp_path):
    path = tmp_path / "bad.json"
    entries = [_entry(tile=300), _entry(ctas_per_sm=-1, len_log2=10), _entry(len_log2=11.5),
               {k: v for k, v in _entry(len_log2=13).items() if k != "stop"},
               _entry(len_log2=14, tile=128), _entry(len_log2=15, variant=2)]
    path.write_text(json.dumps({"entries": entries}))
    capi.serial_emd_tune_load(str(path))
    p = capi.serial_emd_default_params(rows=1, cols=16)
    for L in (1 << 16, 1 << 10, 1 << 13, 1 << 15):
        assert capi.serial_emd_tune_lookup(p, L, 1) is None
    assert capi.serial_emd_tune_lookup(p, 1 << 14, 1) == (128, 2, 0)
    with pytest.raises(capi.SemdError):
        capi.serial_emd_tune_load(str(tmp_path / "missing.json"))
    (tmp_path / "noentries.json").write_text("{}")
    with pytest.raises(capi.SemdError):
        capi.serial_emd_tune_load(str(tmp_path / "noentries.json"))
