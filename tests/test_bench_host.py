"""bench.py's host description of the CPU baseline, on x86-style and Arm-style /proc/cpuinfo."""
import bench


def test_x86_model_name(tmp_path):
    f = tmp_path / "cpuinfo"
    f.write_text("processor\t: 0\nvendor_id\t: GenuineIntel\nmodel name\t: Example CPU @ 2.70GHz\n\n"
                 "processor\t: 1\nmodel name\t: Example CPU @ 2.70GHz\n")
    h = bench.host_cpu(str(f))
    assert h["model"] == "Example CPU @ 2.70GHz" and h["nproc"] >= 1 and h["machine"]


def test_arm_implementer_and_part(tmp_path):
    f = tmp_path / "cpuinfo"
    f.write_text("processor\t: 0\nBogoMIPS\t: 2000.00\nCPU implementer\t: 0x41\nCPU architecture: 8\n"
                 "CPU variant\t: 0x0\nCPU part\t: 0xd4f\n\nprocessor\t: 1\nCPU implementer\t: 0x41\n")
    assert bench.host_cpu(str(f))["model"] == "implementer 0x41 part 0xd4f"


def test_missing_cpuinfo(tmp_path):
    assert bench.host_cpu(str(tmp_path / "absent"))["model"] is None
