"""The benchmark reports the march kernel's DRAM traffic from the committed ncu record only
while the kernel's sources are the ones the record was captured with (a digest of the
listed files); a changed source turns the figure into null instead of a stale number."""
import json
import os
import shutil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _record():
    return json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["k_march_f32"]


def test_record_is_well_formed():
    rec = _record()
    assert rec["dram_bytes_per_launch"] > 0 and 0 < rec["l1_wavefront_frac"] < 1
    assert len(rec["source_digest"]) == 16 and int(rec["source_digest"], 16) >= 0
    assert os.path.exists(os.path.join(ROOT, rec["summary"]))
    for name in rec["sources"]:
        assert os.path.exists(os.path.join(ROOT, "paper_2103_01954_gb300", "csrc", name))


def test_record_used_only_with_matching_sources(tmp_path, monkeypatch):
    import bench
    from paper_2103_01954_gb300 import build as b

    rec = _record()
    # a record stamped with the current sources' digest is reported
    (tmp_path / "profiles").mkdir()
    stamped = dict(rec, source_digest=b.sources_digest(rec["sources"]))
    json.dump({"k_march_f32": stamped}, open(tmp_path / "profiles" / "traffic.json", "w"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._ncu_record("k_march_f32")["dram_bytes_per_launch"] == rec["dram_bytes_per_launch"]
    # one byte appended to one of the kernel's files: the record is dropped
    fake = tmp_path / "csrc"
    shutil.copytree(os.path.join(ROOT, "paper_2103_01954_gb300", "csrc"), fake)
    with open(fake / rec["sources"][0], "a") as f:
        f.write("\n")
    monkeypatch.setattr(b, "CSRC", str(fake))
    assert b.sources_digest(rec["sources"]) != stamped["source_digest"]
    assert bench._ncu_record("k_march_f32") == {}
    # so is a record of an unknown kernel
    assert bench._ncu_record("k_other") == {}
