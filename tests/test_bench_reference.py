"""bench.py --impl reference (the FP64 oracle on the host cores) prints one JSON line
with the reference contract's fields, on slices that hold instrument pixels."""
import argparse
import json


def test_oracle_sample_has_pixels():
    import bench
    from paper_2607_24141_gb300 import inputs as I
    assert I.small_config1(n_lambda_span_nm=2.0, seed=1).instrument.pix_lambda_nm.size > 0
    ev, dt, desc = bench.oracle_sample(span_nm=2.0)
    assert ev > 0 and dt > 0 and "2.0 nm" in desc


def test_reference_arm_prints_one_line(capsys):
    import bench
    args = argparse.Namespace(steps=1, warmup=0, gpus=1)
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == bench.UNIT
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
