"""The bench's profiling aids on synthetic ncu output (CPU): kernel names
map to the kinds the roofline counts, a launch list becomes per-kernel
launches, time per step and shares, and single-kernel counters become
DRAM bytes per launch and per step."""

import json


def test_kernel_kinds():
    import bench
    assert bench.kernel_kind("void ibm::k_slab<256, 8>(float2 *, const float2 *)") == "pencil"
    assert bench.kernel_kind("void ibm::k_rows_fwd_res_s<0, 0>(ibm::ResidualArgs)") == "residual"
    assert bench.kernel_kind("void ibm::k_rows_fwd_t<256>(const float *)") == "forward"
    assert bench.kernel_kind("void ibm::k_rows_inv_t<256>(const float2 *)") == "inverse"
    assert bench.kernel_kind("void ibm::k_cols<float, 256, true>(float2 *)") == "inverse"
    assert bench.kernel_kind("void ibm::k_cols<float, 256, false>(float2 *)") == "forward"
    assert bench.kernel_kind("void at::native::vectorized_elementwise_kernel<4>()") is None


def _launch_csv(path, rows):
    head = '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'
    with open(path, "w") as f:
        f.write("==PROF== a line that is not CSV\n" + head)
        for i, (name, unit, val) in enumerate(rows):
            f.write('"%d","%s","gpu__time_duration.sum","%s","%s"\n' % (i, name, unit, val))


def test_launch_list_summary(tmp_path, capsys):
    import bench
    p = tmp_path / "launches.csv"
    # two steps: two slab launches, one forward launch and a foreign kernel per step
    rows = []
    for _ in range(2):
        rows += [("void ibm::k_slab<256, 8>(x)", "usecond", "60"), ("void ibm::k_slab<256, 8>(x)", "usecond", "60"),
                 ("void ibm::k_rows_fwd_t<256>(x)", "nsecond", "30,000"), ("void other_kernel()", "usecond", "5")]
    _launch_csv(p, rows)
    bench.ncu_summary(str(p), steps=2)
    out = capsys.readouterr().out.splitlines()
    table = {ln.split("|")[1].strip(): [c.strip() for c in ln.split("|")[2:6]] for ln in out[2:]}
    assert table["k_slab<256, 8>"] == ["pencil", "2.0", "120.00", "80.0%"]
    assert table["k_rows_fwd_t<256>"] == ["forward", "1.0", "30.00", "20.0%"]
    assert len(table) == 2  # the foreign kernel is left out


def test_counters_record(tmp_path, monkeypatch):
    import bench
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_digest", lambda kind, which="headline": "digest-" + kind)
    p = tmp_path / "cnt.csv"
    with open(p, "w") as f:
        f.write('"ID","Kernel Name","dram__bytes_read.sum","dram__bytes_write.sum"\n')
        f.write('"","","Mbyte","Kbyte"\n')
        f.write('"0","void ibm::k_rows_inv_t<256>(x)","67.5","6,000"\n')
        f.write('"1","void ibm::k_rows_inv_t<256>(x)","134.5","7,000"\n')
    bench.ncu_counters(str(p), "headline", 2)
    d = json.load(open(tmp_path / "profiles" / "dram_traffic.json"))
    e = d["headline"]["inverse"]
    assert e["dram_bytes_per_launch"] == (67.5e6 + 6e6 + 134.5e6 + 7e6) / 2
    assert e["dram_bytes_per_step"] == 2 * e["dram_bytes_per_launch"]
    assert e["launches_per_step"] == 2 and e["source_sha256_16"] == "digest-inverse"
    # the recorded figure is served only while the sources are unchanged
    assert bench.ncu_traffic("inverse") == e["dram_bytes_per_step"]
    monkeypatch.setattr(bench, "source_digest", lambda kind, which="headline": "changed")
    assert bench.ncu_traffic("inverse") is None


def test_clock_record_and_verdict():
    import bench
    s = bench.ClockSampler(0)
    # index, sm, max sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    s.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2040, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    c = s.summary()
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    assert bench.clock_verdict(c) == {"accepted": True, "why": "sw_power_cap"}
    assert bench.clock_verdict({"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []})["accepted"] is True
    v = bench.clock_verdict({"sm_mhz": 2000.0, "sm_max_mhz": 2070.0, "reasons": ["hw_thermal_slowdown"]})
    assert v == {"accepted": False, "why": "hw_thermal_slowdown"}
    # stuck well below the maximum with no reason: a leftover clock lock
    assert bench.clock_verdict({"sm_mhz": 1400.0, "sm_max_mhz": 2070.0, "reasons": []}) == \
        {"accepted": False, "why": "pinned_low"}
    assert bench.clock_verdict({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]})["accepted"] is None
