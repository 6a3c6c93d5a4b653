"""The JSON files under paper_1910_01031_gb300/configs/ describe exactly the
workloads synth builds (they are written by synth.write_configs), and load
back to equal Config objects."""
import json
import os

from paper_1910_01031_gb300 import synth


def test_config_files_match_the_workloads():
    names = sorted(f[:-5] for f in os.listdir(synth.CONFIG_DIR) if f.endswith(".json"))
    assert names == sorted(synth.workloads())
    for name, cfg in synth.workloads().items():
        assert synth.load_config(name) == cfg, name
        with open(os.path.join(synth.CONFIG_DIR, name + ".json")) as f:
            assert f.read() == synth.config_to_json(cfg), name


def test_round_trip_through_a_file(tmp_path):
    cfg = synth.config1(n_particles=3, seed=99)
    p = tmp_path / "c.json"
    p.write_text(synth.config_to_json(cfg))
    back = synth.load_config(str(p))
    assert back == cfg and back.obs_sigma == cfg.obs_sigma
    assert json.loads(p.read_text())["seed"] == 99
