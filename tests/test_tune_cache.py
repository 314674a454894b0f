"""Host logic of the launch-tuning cache (no GPU): the key separates every
field that changes which tuning is fastest, and the JSON store round-trips,
survives a corrupt file and replaces the file atomically."""
import json

import paper_1602_01410_gb300 as pkg

BASE = dict(shapes=[(1024, 1024)], channels=1, ksize=21, dtype=pkg.DECONV_F32, relax=2.0, kernel_per_image=0,
            ksizes=None, options=(1, 0, 1e-3, 0.0), device="GB300 / 152 SMs")


def test_key_is_stable_and_separates_every_field():
    k0 = pkg.tune_key(**BASE)
    assert k0 == pkg.tune_key(**BASE)
    variants = dict(shapes=[(1024, 1536)], channels=3, ksize=13, dtype=pkg.DECONV_F64, relax=1.0,
                    kernel_per_image=1, ksizes=[21], options=(10, 0, 1e-3, 0.0), device="other / 148 SMs")
    keys = {k0}
    for field, value in variants.items():
        keys.add(pkg.tune_key(**dict(BASE, **{field: value})))
    assert len(keys) == 1 + len(variants)
    assert json.loads(k0)["source"] == pkg._source_digest()


def test_store_round_trip_and_corrupt_file(tmp_path):
    path = str(tmp_path / "tunes.json")
    store = pkg.TuneCache(path)
    assert store.get("k") is None                       # missing file
    tune = {"row_ctas": 608, "col_ctas": 152, "row_stage": 0, "fft_values": 16, "col_fft_values": 32}
    store.put("k", tune, 0.0456)
    store.put("k2", dict(tune, row_ctas=152), 0.05)
    again = pkg.TuneCache(path)
    assert again.get("k") == {"tune": tune, "ms_per_iter": 0.0456}
    assert again.get("k2")["tune"]["row_ctas"] == 152
    assert sorted(p.name for p in tmp_path.iterdir()) == ["tunes.json"]  # no temporary left behind
    (tmp_path / "tunes.json").write_text("{not json")
    assert pkg.TuneCache(path).get("k") is None          # unreadable reads as empty
    pkg.TuneCache(path).put("k", tune, 1.0)
    assert pkg.TuneCache(path).get("k")["ms_per_iter"] == 1.0
