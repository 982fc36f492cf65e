// Host-side file formats around the re-simulator: a reader for the input
// waveforms of a VCD dump (the RTL or gate-level waveforms that drive a
// re-simulation, Section 1) and a writer of SAIF activity files (the
// simulator's output for power analysis, Section 3).  Plain C++, no device
// code; declared in include/gatspi.h.
#include <cctype>
#include <climits>
#include <exception>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <string>
#include <unordered_map>
#include <vector>

#include "gatspi.h"

namespace {

void say(char* err, int32_t err_len, const std::string& msg) {
  if (err && err_len > 0) {
    std::snprintf(err, (size_t)err_len, "%s", msg.c_str());
  }
}

// Whitespace-separated tokens of a whole file.
class Tokens {
 public:
  explicit Tokens(std::string text) : s_(std::move(text)) {}
  bool next(std::string& tok) {
    while (p_ < s_.size() && std::isspace((unsigned char)s_[p_])) ++p_;
    if (p_ >= s_.size()) return false;
    const size_t b = p_;
    while (p_ < s_.size() && !std::isspace((unsigned char)s_[p_])) ++p_;
    tok.assign(s_, b, p_ - b);
    return true;
  }

 private:
  std::string s_;
  size_t p_ = 0;
};

// Picoseconds per unit of a VCD $timescale ("1ps", "10 ns", ...); 0 if the
// unit is below 1 ps or unknown.
int64_t timescale_ps(const std::string& spec) {
  size_t k = 0;
  while (k < spec.size() && std::isdigit((unsigned char)spec[k])) ++k;
  if (k == 0) return 0;
  const int64_t mag = std::stoll(spec.substr(0, k));
  std::string unit = spec.substr(k);
  static const std::pair<const char*, int64_t> units[] = {
      {"s", 1000000000000ll}, {"ms", 1000000000ll}, {"us", 1000000ll}, {"ns", 1000ll}, {"ps", 1ll}};
  if (mag != 1 && mag != 10 && mag != 100) return 0;
  for (const auto& u : units)
    if (unit == u.first) return mag * u.second;
  return 0;
}

int vcd_read(const char* path, int32_t num_names, const char* const* names, uint8_t* init, int32_t* ev_input,
             int64_t* ev_time, int64_t cap, int64_t* num_events, char* err, int32_t err_len) {
  if (!path || num_names < 1 || !names || !init || !num_events || cap < 0 ||
      (cap > 0 && (!ev_input || !ev_time))) {
    say(err, err_len, "bad arguments");
    return GATSPI_EINVAL;
  }
  std::ifstream f(path, std::ios::binary);
  if (!f) {
    say(err, err_len, std::string("cannot open ") + path);
    return GATSPI_EINVAL;
  }
  std::string text((std::istreambuf_iterator<char>(f)), std::istreambuf_iterator<char>());
  Tokens tk(std::move(text));

  // requested names -> input index; a name may be a bare signal name or a
  // dot-separated path from the top scope
  std::unordered_map<std::string, int32_t> want;
  for (int32_t k = 0; k < num_names; ++k) {
    if (!names[k]) {
      say(err, err_len, "null signal name");
      return GATSPI_EINVAL;
    }
    if (!want.emplace(names[k], k).second) {
      say(err, err_len, std::string("signal named twice: ") + names[k]);
      return GATSPI_EINVAL;
    }
  }
  std::vector<int32_t> found_by(num_names, 0);  // how many vars matched each name
  std::unordered_map<std::string, std::vector<int32_t>> code_inputs;  // id code -> inputs
  std::vector<std::string> scope;
  int64_t unit_ps = 1;
  std::string tok;

  // header
  bool defs_done = false;
  while (!defs_done && tk.next(tok)) {
    if (tok == "$timescale") {
      std::string spec, t2;
      while (tk.next(t2) && t2 != "$end") spec += t2;
      unit_ps = timescale_ps(spec);
      if (unit_ps == 0) {
        say(err, err_len, "unsupported $timescale '" + spec + "' (1, 10 or 100 of s, ms, us, ns or ps)");
        return GATSPI_EINVAL;
      }
    } else if (tok == "$scope") {
      std::string kind, name, t2;
      tk.next(kind);
      tk.next(name);
      while (tk.next(t2) && t2 != "$end") {}
      scope.push_back(name);
    } else if (tok == "$upscope") {
      while (tk.next(tok) && tok != "$end") {}
      if (!scope.empty()) scope.pop_back();
    } else if (tok == "$var") {
      std::string type, width, code, ref, t2;
      tk.next(type);
      tk.next(width);
      tk.next(code);
      tk.next(ref);
      while (tk.next(t2) && t2 != "$end") {}
      std::string full;
      for (const auto& s : scope) full += s + ".";
      full += ref;
      for (const std::string* key : {&full, &ref}) {
        auto it = want.find(*key);
        if (it == want.end()) continue;
        if (width != "1") {
          say(err, err_len, "signal " + *key + " is " + width + " bits wide; inputs are 1-bit nets");
          return GATSPI_EINVAL;
        }
        code_inputs[code].push_back(it->second);
        found_by[it->second]++;
        break;
      }
    } else if (tok == "$enddefinitions") {
      while (tk.next(tok) && tok != "$end") {}
      defs_done = true;
    } else if (tok.size() > 1 && tok[0] == '$') {  // $date, $version, $comment, ...
      while (tk.next(tok) && tok != "$end") {}
    }
  }
  if (!defs_done) {
    say(err, err_len, "no $enddefinitions");
    return GATSPI_EINVAL;
  }
  for (int32_t k = 0; k < num_names; ++k) {
    if (found_by[k] == 0) {
      say(err, err_len, std::string("signal not in the dump: ") + names[k]);
      return GATSPI_EINVAL;
    }
    if (found_by[k] > 1) {
      say(err, err_len, std::string("signal name is ambiguous: ") + names[k]);
      return GATSPI_EINVAL;
    }
  }

  // value changes: an input's first value, at time 0, is its initial value;
  // every time step (time 0 included) whose final value differs from the
  // value before the step is a toggle at that time
  std::vector<int8_t> cur(num_names, -1), committed(num_names, -1), first(num_names, -1);
  std::vector<int32_t> touched;
  std::vector<uint8_t> is_touched(num_names, 0);
  int64_t now = 0, count = 0;
  bool have_time = false;
  auto commit = [&]() {
    for (int32_t k : touched) {
      is_touched[k] = 0;
      if (cur[k] != committed[k]) {
        if (count < cap) {
          ev_input[count] = k;
          ev_time[count] = now * unit_ps;
        }
        ++count;
        committed[k] = cur[k];
      }
    }
    touched.clear();
  };
  bool dump_off = false;  // inside a $dumpoff block: its (x) values are not changes
  auto change = [&](char v, const std::string& code) -> int {
    auto it = code_inputs.find(code);
    if (it == code_inputs.end()) return GATSPI_OK;  // not an input of interest
    if (dump_off) return GATSPI_OK;
    if (v != '0' && v != '1') {
      say(err, err_len, std::string("value '") + v + "' at time " + std::to_string(now) +
                            ": the simulation is 2-valued (0/1)");
      return GATSPI_EINVAL;
    }
    if (!have_time) {
      say(err, err_len, "value change before the first #time");
      return GATSPI_EINVAL;
    }
    for (int32_t k : it->second) {
      if (committed[k] < 0) {  // the first value: the initial one, at time 0 only
        if (now != 0) {
          say(err, err_len, std::string("the first value of ") + names[k] + " comes after time 0");
          return GATSPI_EINVAL;
        }
        first[k] = committed[k] = cur[k] = (int8_t)(v - '0');
        continue;
      }
      cur[k] = (int8_t)(v - '0');
      if (!is_touched[k]) {
        is_touched[k] = 1;
        touched.push_back(k);
      }
    }
    return GATSPI_OK;
  };
  while (tk.next(tok)) {
    const char c0 = tok[0];
    if (c0 == '#') {
      const std::string num = tok.substr(1);
      if (num.empty() || num.find_first_not_of("0123456789") != std::string::npos) {
        say(err, err_len, "bad time '" + tok + "'");
        return GATSPI_EINVAL;
      }
      if (num.size() > 18) {  // keeps the time, and the time in ps, inside int64
        say(err, err_len, "time too large: '" + tok + "'");
        return GATSPI_EINVAL;
      }
      const int64_t t = std::stoll(num);
      if (t > INT64_MAX / unit_ps) {
        say(err, err_len, "time too large in ps: '" + tok + "'");
        return GATSPI_EINVAL;
      }
      if (have_time && t < now) {
        say(err, err_len, "time goes back at '" + tok + "'");
        return GATSPI_EINVAL;
      }
      if (have_time && t != now) commit();
      if (!have_time && t != 0) {
        say(err, err_len, "the dump must start at #0");
        return GATSPI_EINVAL;
      }
      now = t;
      have_time = true;
    } else if (c0 == '$') {
      // $dumpvars / $dumpall / $dumpon / $end: value changes inside them
      // count as ordinary changes.  $dumpoff lists every variable as x
      // until its $end: those are no changes (the waveform is not dumped
      // until $dumpon, whose values then count as changes at its time).
      // Other commands are skipped.
      if (tok == "$comment") {
        while (tk.next(tok) && tok != "$end") {}
      } else if (tok == "$dumpoff") {
        dump_off = true;
      } else if (tok == "$end") {
        dump_off = false;
      }
    } else if (c0 == '0' || c0 == '1' || c0 == 'x' || c0 == 'X' || c0 == 'z' || c0 == 'Z') {
      int rc = change(c0, tok.substr(1));
      if (rc) return rc;
    } else if (c0 == 'b' || c0 == 'B') {
      std::string code;
      tk.next(code);
      if (code_inputs.count(code)) {
        const std::string bits = tok.substr(1);
        if (bits.size() != 1) {
          say(err, err_len, "vector value for a 1-bit input");
          return GATSPI_EINVAL;
        }
        int rc = change(bits[0], code);
        if (rc) return rc;
      }
    } else if (c0 == 'r' || c0 == 'R') {
      std::string code;
      tk.next(code);  // real values: never an input of interest
    }
  }
  if (have_time) commit();
  for (int32_t k = 0; k < num_names; ++k) {
    if (first[k] < 0) {
      say(err, err_len, std::string("no value at time 0 for ") + names[k]);
      return GATSPI_EINVAL;
    }
    init[k] = (uint8_t)first[k];
  }
  *num_events = count;
  if (count > cap) {
    say(err, err_len, "event buffers too small: need " + std::to_string(count));
    return GATSPI_ECAPACITY;
  }
  return GATSPI_OK;
}

}  // namespace

extern "C" {

// The parser reads untrusted files behind a C interface: no exception may
// leave it.
int gatspi_vcd_read(const char* path, int32_t num_names, const char* const* names, uint8_t* init,
                    int32_t* ev_input, int64_t* ev_time, int64_t cap, int64_t* num_events, char* err,
                    int32_t err_len) {
  try {
    return vcd_read(path, num_names, names, init, ev_input, ev_time, cap, num_events, err, err_len);
  } catch (const std::exception& e) {
    say(err, err_len, std::string("VCD read failed: ") + e.what());
    return GATSPI_EINVAL;
  } catch (...) {
    say(err, err_len, "VCD read failed");
    return GATSPI_EINVAL;
  }
}

int gatspi_saif_write(const char* path, const char* design, int64_t duration_ps, int32_t num_nets,
                      const char* const* net_names, const int64_t* t0, const int64_t* t1, const int64_t* tc,
                      char* err, int32_t err_len) {
  if (!path || !design || num_nets < 0 || (num_nets > 0 && (!net_names || !t0 || !t1 || !tc)) ||
      duration_ps < 0) {
    say(err, err_len, "bad arguments");
    return GATSPI_EINVAL;
  }
  // SAIF identifiers: characters other than letters, digits and '_' are
  // escaped with a backslash
  auto ident = [](const char* s) {
    std::string o;
    for (const char* p = s; *p; ++p) {
      if (!(std::isalnum((unsigned char)*p) || *p == '_')) o += '\\';
      o += *p;
    }
    return o;
  };
  std::FILE* f = std::fopen(path, "w");
  if (!f) {
    say(err, err_len, std::string("cannot write ") + path);
    return GATSPI_EINVAL;
  }
  std::fprintf(f, "(SAIFILE\n(SAIFVERSION \"2.0\")\n(DIRECTION \"backward\")\n(DESIGN \"%s\")\n", design);
  std::fprintf(f, "(PROGRAM_NAME \"gatspi-gb300\")\n(DIVIDER / )\n(TIMESCALE 1 ps)\n");
  std::fprintf(f, "(DURATION %lld)\n(INSTANCE %s\n  (NET\n", (long long)duration_ps, ident(design).c_str());
  for (int32_t n = 0; n < num_nets; ++n) {
    if (!net_names[n]) {
      std::fclose(f);
      say(err, err_len, "null net name");
      return GATSPI_EINVAL;
    }
    std::fprintf(f, "    (%s\n      (T0 %lld) (T1 %lld) (TX 0)\n      (TC %lld) (IG 0)\n    )\n",
                 ident(net_names[n]).c_str(), (long long)t0[n], (long long)t1[n], (long long)tc[n]);
  }
  std::fprintf(f, "  )\n)\n)\n");
  if (std::fclose(f) != 0) {
    say(err, err_len, std::string("write failed: ") + path);
    return GATSPI_EINVAL;
  }
  return GATSPI_OK;
}

}  // extern "C"
